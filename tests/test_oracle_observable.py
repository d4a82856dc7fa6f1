"""Pins of the oracle's observable histogram (the p_T distribution of the
first final-state particle, filled during the VEGAS passes): the bins add up
to the pass sums, a brute-force refill from per-event outputs reproduces
them, one all-covering bin is the cross section itself, and for g g -> t tbar
(no cuts, fixed scale) the combined histogram agrees with a deterministic
quadrature of the closed-form partonic cross section over each p_T bin."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from tests.test_oracle_integration import sig_hat_gg

PB = 0.3893793721e9


def test_obs_bins_add_up_to_pass_sums():
    ph = IN.Physics(seed=2)
    pdf = O.Pdf(IN.make_pdf_grid())
    for proc in (IN.GG_TT, IN.GG_TTG, IN.UU_TT):
        g = O.vegas_init(IN.DIM[proc], 50)
        r = O.vegas_pass_obs(proc, ph, pdf, g, 4000, 12, 20.0, 500.0, iteration=1)
        assert r["obs"][:, 0].sum() == pytest.approx(r["sum_w"], rel=1e-13, abs=0.0)
        assert r["obs"][:, 1].sum() == pytest.approx(r["sum_w2"], rel=1e-13, abs=0.0)
        # the same pass without the observable gives the same sums
        p = O.vegas_pass(proc, ph, pdf, g, 4000, iteration=1)
        assert p["sum_w"] == r["sum_w"] and p["sum_w2"] == r["sum_w2"]


def test_obs_matches_brute_force_refill():
    """Per-event outputs binned in Python: p_T from the partonic momenta (the
    lab boost is longitudinal), bin by the definition, weights w/N."""
    ph = IN.Physics(seed=5)
    pdf = O.Pdf(IN.make_pdf_grid())
    proc, n, nobs, lo, hi = IN.GG_TTG, 400, 7, 50.0, 400.0
    g = O.vegas_init(IN.DIM[proc], 50)
    r = O.vegas_pass_obs(proc, ph, pdf, g, n, nobs, lo, hi, iteration=2)
    ref = np.zeros((nobs + 2, 2))
    for e in range(n):
        o = O.event(proc, ph, pdf, g, e, 2)
        pt = math.hypot(o.plab[9], o.plab[10])          # particle 2 in the lab: px, py
        if pt < lo:
            j = 0
        elif pt >= hi:
            j = nobs + 1
        else:
            j = 1 + int(math.floor((pt - lo) / (hi - lo) * nobs))
        edge = min(abs((pt - lo) / (hi - lo) * nobs - k) for k in range(nobs + 1))
        assert edge > 1e-9, "event on a bin edge"
        assert O.obs_bin(o.p[9], o.p[10], nobs, lo, hi) == j
        ref[j, 0] += o.w / n
        ref[j, 1] += (o.w / n) ** 2
    assert np.allclose(r["obs"], ref, rtol=1e-12, atol=0.0)


def test_obs_bin_edges_and_specials():
    assert O.obs_bin(0.0, 0.0, 4, 10.0, 50.0) == 0
    assert O.obs_bin(10.0, 0.0, 4, 10.0, 50.0) == 1      # lower edge of the first bin
    assert O.obs_bin(0.0, -20.0, 4, 10.0, 50.0) == 2     # 20 GeV: second bin
    assert O.obs_bin(49.999, 0.0, 4, 10.0, 50.0) == 4
    assert O.obs_bin(50.0, 0.0, 4, 10.0, 50.0) == 5      # upper edge: overflow
    assert O.obs_bin(float("nan"), 0.0, 4, 10.0, 50.0) == 0
    assert O.obs_bin(float("inf"), 0.0, 4, 10.0, 50.0) == 5


def test_one_covering_bin_is_the_cross_section():
    ph = IN.Physics(seed=1)
    pdf = O.Pdf(IN.make_pdf_grid())
    r = O.integrate_obs(IN.GG_TT, ph, pdf, 20000, 3, 1, 0.0, 1e9)
    ref = O.integrate(IN.GG_TT, ph, pdf, 20000, 3)
    assert r["sigma"] == ref["sigma"]
    assert r["hist"][0] == 0.0 and r["hist"][2] == 0.0
    assert r["hist"][1] == pytest.approx(ref["sigma"], rel=1e-13)
    assert r["err"][1] == pytest.approx(ref["error"], rel=1e-9)


def sigma_hat_bin_gg(ph, s, a, b, n=48):
    """Partonic g g -> t tbar cross section with a <= p_T(t) < b at shat = s:
    d sigma/d cos = |M|^2 beta / (32 pi s) over the cos(theta) range of the bin."""
    m = ph.mt
    E = 0.5 * math.sqrt(s)
    if E <= m:
        return 0.0
    p = math.sqrt(E * E - m * m)
    beta = p / E
    if a >= p:
        return 0.0
    c2 = math.sqrt(max(0.0, 1.0 - (a / p) ** 2))
    c1 = math.sqrt(max(0.0, 1.0 - (b / p) ** 2)) if b < p else 0.0
    gs = math.sqrt(4 * math.pi * ph.alpha_s)
    xg, wg = np.polynomial.legendre.leggauss(n)
    tot = 0.0
    for x, w in zip(xg, wg):
        c = 0.5 * (c2 - c1) * x + 0.5 * (c2 + c1)
        for cs in (c, -c):
            sn = math.sqrt(max(0.0, 1.0 - cs * cs))
            mom = np.array([[E, 0, 0, E], [E, 0, 0, -E], [E, p * sn, 0, p * cs], [E, -p * sn, 0, -p * cs]])
            tot += 0.5 * (c2 - c1) * w * O.me2_gg_tt_closed(m, gs, mom) * beta / (32 * math.pi * s)
    return tot


def test_bin_quadrature_reproduces_closed_form_sigma_hat():
    """The p_T-bin integrals over [0, inf) add up to the closed-form sigma_hat."""
    ph = IN.Physics(seed=1)
    f = sig_hat_gg(ph)
    for rs in (400.0, 1000.0, 3000.0):
        s = rs * rs
        edges = [0.0, 50.0, 150.0, 300.0, 1e9]
        tot = sum(sigma_hat_bin_gg(ph, s, edges[i], edges[i + 1]) for i in range(len(edges) - 1))
        assert tot == pytest.approx(f(s), rel=1e-6), rs


def hadronic_bins_quadrature(ph, pdf, edges, n=40, ny=96):
    """sigma_j = int dtau dy g(x1) g(x2)/(x1 x2) sigma_hat_j(tau S) at mu_F = m_t.
    ln tau is split where p(shat) crosses a bin edge (a bin switches on there
    like a square root); on each piece ln tau = L_a + (L_b - L_a) v^2 removes
    that onset, and v takes n Gauss-Legendre points."""
    S = ph.sqrt_s ** 2
    m2 = ph.mt ** 2
    lt0 = math.log(4 * m2 / S)
    q2 = m2
    xv, wv = np.polynomial.legendre.leggauss(n)
    xy, wy = np.polynomial.legendre.leggauss(ny)
    brk = sorted({lt0, 0.0} | {math.log(4 * (e * e + m2) / S) for e in edges
                               if 0.0 < e and 4 * (e * e + m2) < S})
    out = np.zeros(len(edges) - 1)
    for La, Lb in zip(brk[:-1], brk[1:]):
        for x, w in zip(xv, wv):
            v = 0.5 * (x + 1)
            lt = La + (Lb - La) * v * v
            jac = 0.5 * w * 2 * (Lb - La) * v
            tau = math.exp(lt)
            ymax = -0.5 * lt
            lum = 0.0
            for b_, wb in zip(xy, wy):
                y = b_ * ymax
                x1 = math.sqrt(tau) * math.exp(y); x2 = math.sqrt(tau) * math.exp(-y)
                lum += wb * ymax * pdf.xf(0, x1, q2) / x1 * pdf.xf(0, x2, q2) / x2
            pre = jac * tau * lum
            for j in range(len(edges) - 1):
                out[j] += pre * sigma_hat_bin_gg(ph, tau * S, edges[j], edges[j + 1], n=24)
    return out * PB


def test_bins_quadrature_converged_and_adds_up():
    """The piecewise quadrature is converged (n = 40 against 80 points a piece)
    and its bins add up to the plain hadronic quadrature of the closed-form
    sigma_hat."""
    from tests.test_oracle_integration import sigma_hadronic_quadrature
    ph = IN.Physics(seed=1)
    pdf = O.Pdf(IN.make_pdf_grid())
    edges = [0.0, 100.0, 200.0, 300.0, 1e9]
    a = hadronic_bins_quadrature(ph, pdf, edges, n=40, ny=64)
    b = hadronic_bins_quadrature(ph, pdf, edges, n=80, ny=64)
    assert np.allclose(a, b, rtol=1e-5, atol=0.0), (a, b)
    ref = sigma_hadronic_quadrature(ph, pdf, sig_hat_gg(ph), 0, 0, n=160)
    assert a.sum() == pytest.approx(ref, rel=5e-4)


def test_gg_tt_pt_distribution_matches_quadrature():
    """The oracle's combined p_T histogram of g g -> t tbar (5 iterations of
    1e5 events) against the quadrature, bin by bin within 4 standard errors."""
    ph = IN.Physics(seed=1)
    pdf = O.Pdf(IN.make_pdf_grid())
    nobs, lo, hi = 6, 0.0, 300.0
    r = O.integrate_obs(IN.GG_TT, ph, pdf, 100_000, 5, nobs, lo, hi)
    edges = [lo + (hi - lo) * k / nobs for k in range(nobs + 1)] + [1e9]
    q = hadronic_bins_quadrature(ph, pdf, edges)
    assert r["hist"][0] == 0.0
    pulls = []
    for j in range(nobs + 1):
        h, e = r["hist"][j + 1], r["err"][j + 1]
        assert abs(h - q[j]) < 4 * e, (j, h, e, q[j])
        assert e < 0.05 * q[j]
        pulls.append((h - q[j]) / e)
    assert sum(p * p for p in pulls) / len(pulls) < 3.0, pulls
    assert r["hist"].sum() == pytest.approx(r["sigma"], rel=1e-12)

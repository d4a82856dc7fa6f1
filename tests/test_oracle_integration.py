"""End-to-end pins of the oracle's Monte Carlo pipeline (Philox -> VEGAS ->
phase space -> PDF -> |M|^2 -> weight -> iterations): its cross sections must
agree, within the stated MC error, with deterministic quadratures built from
closed forms that are pinned on their own in test_oracle_pins.py."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN

PB = 0.3893793721e9


def sigma_ee_quadrature(ph):
    s = ph.sqrt_s ** 2
    E = ph.sqrt_s / 2
    xg, wg = np.polynomial.legendre.leggauss(40)
    tot = 0.0
    for c, w in zip(xg, wg):
        sn = math.sqrt(1 - c * c)
        p = np.array([[E, 0, 0, E], [E, 0, 0, -E], [E, E * sn, 0, E * c], [E, -E * sn, 0, -E * c]])
        tot += w * O.me2_ee_mumu_closed(ph, p) / (32 * math.pi * s)
    return tot * PB


def sigma_hadronic_quadrature(ph, pdf, sig_hat, f1, f2, n=160):
    """sigma = int dtau dy f1(sqrt(tau) e^y) f2(sqrt(tau) e^-y) sigma_hat(tau S) at mu_F = m_t."""
    S = ph.sqrt_s ** 2
    tau0 = 4 * ph.mt ** 2 / S
    xg, wg = np.polynomial.legendre.leggauss(n)
    lt0 = math.log(tau0)
    tot = 0.0
    q2 = ph.mt ** 2
    for a, wa in zip(xg, wg):
        lt = 0.5 * (a + 1) * lt0                  # ln tau in [ln tau0, 0]
        tau = math.exp(lt)
        ymax = -0.5 * lt
        sh = sig_hat(tau * S)
        inner = 0.0
        for b, wb in zip(xg, wg):
            y = b * ymax
            x1 = math.sqrt(tau) * math.exp(y); x2 = math.sqrt(tau) * math.exp(-y)
            inner += wb * ymax * pdf.xf(f1, x1, q2) / x1 * pdf.xf(f2, x2, q2) / x2
        tot += wa * 0.5 * (-lt0) * tau * inner * sh
    return tot * PB


def sig_hat_gg(ph):
    a_s = ph.alpha_s

    def f(s):
        rho = 4 * ph.mt ** 2 / s
        beta = math.sqrt(max(1 - rho, 0.0))
        if beta <= 0:
            return 0.0
        return math.pi * a_s ** 2 / (3 * s) * ((1 + rho + rho * rho / 16) * math.log((1 + beta) / (1 - beta))
                                               - beta * (7 / 4 + 31 * rho / 16))
    return f


def sig_hat_qq(ph):
    a_s = ph.alpha_s

    def f(s):
        rho = 4 * ph.mt ** 2 / s
        beta = math.sqrt(max(1 - rho, 0.0))
        return 8 * math.pi * a_s ** 2 / (27 * s) * beta * (1 + rho / 2)
    return f


def test_ee_mumu_vegas_matches_quadrature():
    ph = IN.Physics(sqrt_s=91.19, seed=0)
    pdf = O.Pdf(IN.make_pdf_grid())
    r = O.integrate(IN.EE_MUMU, ph, pdf, 100_000, 5)
    ref = sigma_ee_quadrature(ph)
    assert abs(r["sigma"] - ref) < 4 * r["error"], (r, ref)
    assert r["error"] < 1e-4 * ref


@pytest.mark.parametrize("proc", [IN.GG_TT, IN.UU_TT])
def test_tt_vegas_matches_quadrature(proc):
    ph = IN.Physics(seed=1)
    pdf = O.Pdf(IN.make_pdf_grid())
    n = 100_000 if proc == IN.GG_TT else 50_000
    r = O.integrate(proc, ph, pdf, n, 5)
    if proc == IN.GG_TT:
        ref = sigma_hadronic_quadrature(ph, pdf, sig_hat_gg(ph), 0, 0)
    else:
        ref = sigma_hadronic_quadrature(ph, pdf, sig_hat_qq(ph), 1, 2)
    assert abs(r["sigma"] - ref) < 4 * r["error"], (r, ref)
    assert r["error"] < 5e-3 * ref


def test_alpha_s_scaling_exact():
    """sigma is proportional to alpha_s^k (no running): d sigma / d alpha_s = k sigma / alpha_s;
    at fixed random numbers the estimator scales exactly."""
    pdf = O.Pdf(IN.make_pdf_grid())
    grid = O.vegas_init(14, 50)
    a = O.vegas_pass(IN.GG_TTG, IN.Physics(seed=2), pdf, grid, 300)
    b = O.vegas_pass(IN.GG_TTG, IN.Physics(seed=2, alpha_s=0.118 * 1.1), pdf, grid, 300)
    assert abs(b["sum_w"] / a["sum_w"] - 1.1 ** 3) < 1e-12

"""Helicity sums (Sec. 2.2: the generated matrix element loops over the
helicity configurations and adds their contributions).  The per-helicity
profile (mf_helicity_profile) is the measurement behind two shortcuts of the
integrand: configurations that helicity conservation on a massless quark or
lepton line forbids are skipped (they must vanish exactly), and of every pair
of parity mirrors in the gluon processes only one is evaluated and doubled
(the pair must agree).  Each row of the profile must add up to the |M|^2 of
mf_evaluate and of the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from tests.gpu_common import EPS, PHYS, me_condition, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROCS = [IN.EE_MUMU, IN.GG_TT, IN.GG_TTG, IN.GG_TTGG, IN.UU_TT, IN.UG_TTU]
# helicity bit rules of the massless lines: (bit a, bit b, same) -> bits a and b equal (same) or opposite
MASSLESS_RULES = {IN.EE_MUMU: [(0, 1, False), (2, 3, False)], IN.UU_TT: [(0, 1, False)], IN.UG_TTU: [(0, 4, True)]}


def points(proc, n_per_shat, seed):
    phys = PHYS[proc]
    rng = np.random.default_rng(seed)
    n_ext = IN.N_EXT[proc]
    nf = n_ext - 2
    masses = [0.0, 0.0] if proc == IN.EE_MUMU else [phys.mt, phys.mt] + [0.0] * (nf - 2)
    moms = []
    for shat_tev2 in (0.5, 1.0, 3.0, 13.0):
        rs = math.sqrt(shat_tev2) * 1000.0 if proc != IN.EE_MUMU else 91.19 * shat_tev2
        for _ in range(n_per_shat):
            pf, _ = O.rambo(nf, rs, masses, rng.random(4 * nf))
            moms.append(np.vstack([[[rs / 2, 0, 0, rs / 2], [rs / 2, 0, 0, -rs / 2]], pf]))
    return np.array(moms)


def allowed(proc, ih):
    for a, b, same in MASSLESS_RULES.get(proc, []):
        if ((ih >> a) & 1 == (ih >> b) & 1) != same:
            return False
    return True


@pytest.mark.parametrize("proc", PROCS)
@pytest.mark.parametrize("prec", [0, 1])
def test_profile_adds_up_and_forbidden_helicities_vanish(proc, prec):
    from paper_2105_10529_gb300.api import Context
    phys = PHYS[proc]
    moms = points(proc, 8, 300 + proc)
    ctx = Context(phys, IN.make_pdf_grid(), precision=prec)
    mt = torch.tensor(moms, device="cuda")
    prof = ctx.helicity_profile(proc, mt).cpu().numpy()
    me = ctx.evaluate(proc, mt).cpu().numpy()
    ctx.close()
    nhel = 1 << IN.N_EXT[proc]
    assert prof.shape == (len(moms), nhel)
    # rows add up to evaluate's |M|^2 (which sums one of each parity pair twice, and skips the
    # forbidden configurations) and, in FP64, to the oracle's
    tol = 1e-13 if prec == 0 else 2e-6
    assert np.all(rel_err(prof.sum(1), me) < tol), float(rel_err(prof.sum(1), me).max())
    if prec == 0:
        ref = np.array([O.me2(proc, phys, p) for p in moms])
        bound = np.array([max(1e-12, 64 * EPS * me_condition(proc, phys, p)) for p in moms])
        assert np.all(rel_err(prof.sum(1), ref) <= bound)
    forb = np.array([not allowed(proc, ih) for ih in range(nhel)])
    if forb.any():
        assert np.all(prof[:, forb] == 0.0)                  # exactly: massless spinors have exact chirality
        assert np.all(prof[:, ~forb].max(0) > 0.0)           # and the allowed ones contribute
        assert forb.sum() == {IN.EE_MUMU: 12, IN.UU_TT: 8, IN.UG_TTU: 16}[proc]
    assert np.all(prof >= 0.0)


@pytest.mark.parametrize("proc", [IN.GG_TT, IN.GG_TTG, IN.GG_TTGG])
def test_parity_mirrors_agree(proc):
    """|M_h|^2 = |M_-h|^2 helicity by helicity (FP64, relative to the row's
    largest entry): the identity behind the gluon processes' parity-halved
    helicity loops."""
    from paper_2105_10529_gb300.api import Context
    phys = PHYS[proc]
    moms = points(proc, 6, 400 + proc)
    ctx = Context(phys, IN.make_pdf_grid(), precision=0)
    prof = ctx.helicity_profile(proc, torch.tensor(moms, device="cuda")).cpu().numpy()
    ctx.close()
    nhel = prof.shape[1]
    mirror = prof[:, [ih ^ (nhel - 1) for ih in range(nhel)]]
    scale = prof.max(1, keepdims=True)
    assert np.all(np.abs(prof - mirror) <= 1e-12 * scale)

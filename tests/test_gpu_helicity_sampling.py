"""Helicity sampling in the g g -> t tbar g g g integrand (the paper's
matrix element sums every helicity configuration, Sec. 2.2; sampling a
stratified subset of them per event keeps the Monte Carlo's expectation and
trades variance for cost).  Three checks through the C ABI:

* the selection: each event's sampled |M|^2 is the weighted sum of exactly
  the configurations that the documented Philox draws pick, taken from the
  per-helicity profile of the same momenta (the draws are restated here from
  the published Philox4x32-10 definition in the oracle);
* unbiasedness: over many independent draw streams on the same events the
  average of the sampled |M|^2 converges to the full sum, with the spread the
  stratified estimator's variance (computed from the profile) predicts;
* the integral: sigma with sampling agrees with sigma without it within the
  Monte Carlo errors."""
import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from tests.gpu_common import random_grid, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROC = IN.GG_TTGGG
PHYS = IN.Physics(seed=6)
HALF = 64   # parity-halved configurations: 2j + 1 stands for the pair {2j + 1, 126 - 2j}


def drawn_configurations(ev, iteration, n_samples, stream, phys=PHYS):
    """Configurations (bit i = helicity of particle i) that event ev draws:
    stratum s of 64 / n_samples consecutive odd configurations, the offset
    inside it from bits [s b, (s + 1) b) of the Philox4x32-10 output words
    (x lowest) at counter (ev lo, ev hi, iteration, channel << 8 | 0xFF), key
    (seed lo ^ 0x68656C69 ^ stream, seed hi)."""
    key = ((phys.seed & 0xFFFFFFFF) ^ 0x68656C69 ^ stream, (phys.seed >> 32) & 0xFFFFFFFF)
    words = O.philox((ev & 0xFFFFFFFF, ev >> 32, iteration, (phys.channel << 8) | 0xFF), key)
    bits = sum(int(w) << (32 * i) for i, w in enumerate(words))
    ssize = HALF // n_samples
    b = ssize.bit_length() - 1
    return [1 + 2 * (s * ssize + ((bits >> (s * b)) & (ssize - 1))) for s in range(n_samples)]


def sampled_from_profile(prof_row, configs):
    ssize = HALF // len(configs)
    return sum(2.0 * ssize * prof_row[ih] for ih in configs)


def ctx_for(prec, pdf_grid):
    from paper_2105_10529_gb300.api import Context
    return Context(PHYS, pdf_grid, precision=prec)


@pytest.fixture(scope="module")
def pdf_grid():
    return IN.make_pdf_grid()


def test_arguments(pdf_grid):
    from paper_2105_10529_gb300._lib import MfError
    ctx = ctx_for(1, pdf_grid)
    for bad in (-1, 3, 6, 65, 128):
        with pytest.raises(MfError):
            ctx.set_helicity_sampling(bad)
    for good in (0, 1, 2, 4, 8, 16, 32, 64):
        ctx.set_helicity_sampling(good)
    ctx.close()


@pytest.mark.parametrize("prec,n_samples,stream", [(0, 4, 7), (0, 1, 0), (1, 8, 3), (1, 32, 11)])
def test_selection_matches_the_documented_draws(prec, n_samples, stream, pdf_grid):
    n, iteration = 173, 2
    grid = torch.tensor(random_grid(IN.DIM[PROC], seed=68), device="cuda")
    ctx = ctx_for(prec, pdf_grid)
    _, full = ctx.vegas_pass(PROC, PHYS.sqrt_s, grid, n, iteration=iteration, want_events=True)
    ctx.set_helicity_sampling(n_samples, stream)
    _, samp = ctx.vegas_pass(PROC, PHYS.sqrt_s, grid, n, iteration=iteration, want_events=True)
    ctx.set_helicity_sampling(0)
    # the events themselves are untouched by the sampling
    for f in ("u", "x", "bins", "mask", "momenta"):
        assert torch.equal(full[f], samp[f]), f
    mask = samp["mask"].cpu().numpy().astype(bool)
    assert mask.sum() > n // 4
    prof = ctx.helicity_profile(PROC, samp["momenta"][torch.tensor(mask, device="cuda")]).cpu().numpy()
    ctx.close()
    me_full = full["me2"].cpu().numpy()[mask]
    me_samp = samp["me2"].cpu().numpy()[mask]
    idx = np.nonzero(mask)[0]
    want = np.array([sampled_from_profile(prof[k], drawn_configurations(int(e), iteration, n_samples, stream))
                     for k, e in enumerate(idx)])
    tol = 1e-12 if prec == 0 else 2e-5
    assert np.all(rel_err(prof.sum(1), me_full) < tol)
    assert np.all(rel_err(me_samp, want) < tol), float(rel_err(me_samp, want).max())
    # the weights carry the estimate: w_sampled / w_full = |M|^2_sampled / |M|^2_full
    w_full = full["w"].cpu().numpy()[mask]
    w_samp = samp["w"].cpu().numpy()[mask]
    assert np.all(rel_err(w_samp * me_full, w_full * me_samp) < (1e-12 if prec == 0 else 1e-5))
    # and the sampled values do differ from the full sum (the selection is not a no-op)
    assert np.mean(rel_err(me_samp, me_full) > 1e-3) > 0.5


def test_unbiased_over_streams(pdf_grid):
    """One configuration per event (the largest variance), M streams on the
    same events: t_e = (mean_e - full_e) / sqrt(var_e / M) with the exact
    per-event variance from the profile; sum t_e and sum t_e^2 as for
    independent standard normals."""
    n, iteration, m = 240, 5, 64
    grid = torch.tensor(random_grid(IN.DIM[PROC], seed=69), device="cuda")
    ctx = ctx_for(0, pdf_grid)
    _, full = ctx.vegas_pass(PROC, PHYS.sqrt_s, grid, n, iteration=iteration, want_events=True,
                             fields=("mask", "me2", "momenta"))
    mask = full["mask"].cpu().numpy().astype(bool)
    runs = []
    for s in range(m):
        ctx.set_helicity_sampling(1, 1000 + s)
        _, ev = ctx.vegas_pass(PROC, PHYS.sqrt_s, grid, n, iteration=iteration, want_events=True,
                               fields=("me2",))
        runs.append(ev["me2"].cpu().numpy()[mask])
    prof = ctx.helicity_profile(PROC, full["momenta"][torch.tensor(mask, device="cuda")]).cpu().numpy()
    ctx.close()
    runs = np.array(runs)
    me_full = full["me2"].cpu().numpy()[mask]
    # one draw: 128 p_h with h uniform over the 64 odd configurations
    vals = 128.0 * prof[:, 1::2]
    assert np.all(rel_err(vals.mean(1), me_full) < 1e-12)
    var = vals.var(1)
    t = (runs.mean(0) - me_full) / np.sqrt(var / m)
    k = len(t)
    assert k > n // 4
    assert abs(t.sum()) < 5.0 * np.sqrt(k), float(t.sum())
    assert 0.6 * k < float((t * t).sum()) < 1.5 * k, float((t * t).sum())


def test_sigma_agrees_with_the_full_sum(pdf_grid):
    n, it = 20000, 3
    ctx = ctx_for(1, pdf_grid)
    full = ctx.integrate(PROC, PHYS.sqrt_s, n, it)
    ctx.set_helicity_sampling(8, 1)
    samp = ctx.integrate(PROC, PHYS.sqrt_s, n, it)
    ctx.set_helicity_sampling(0)
    again = ctx.integrate(PROC, PHYS.sqrt_s, n, it)
    ctx.close()
    assert again["sigma"] == full["sigma"]            # switching it off restores the full sum
    assert samp["sigma"] != full["sigma"]
    d = abs(samp["sigma"] - full["sigma"])
    assert d < 5.0 * np.hypot(samp["error"], full["error"]), (samp, full)

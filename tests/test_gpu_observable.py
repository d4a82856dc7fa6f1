"""GPU parity of the observable histogram (p_T of the first final-state
particle, filled inside the fused integrand) against the FP64 oracle on the
same seeded events: per bin within 1e-11 (FP64 path) and 2e-5 (mixed path)
relative, its Monte Carlo errors likewise, the bins adding up to sigma, and
sigma itself unchanged by switching the histogram on."""
import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from tests.gpu_common import PHYS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# events per pass: light kernels several rounds per CTA; heavy ones several
# matrix-element batches per CTA and a ragged tail
N_OBS = {IN.EE_MUMU: 20011, IN.GG_TT: 50021, IN.UU_TT: 20011, IN.UG_TTU: 20011, IN.GG_TTG: 100003}
SPEC = {IN.EE_MUMU: (10, 0.0, 50.0)}
DEFAULT_SPEC = (12, 0.0, 480.0)
TOL = {0: 1e-11, 1: 2e-5}


@pytest.fixture(scope="module")
def pdf_grid():
    return IN.make_pdf_grid()


@pytest.fixture(scope="module")
def opdf(pdf_grid):
    return O.Pdf(pdf_grid)


_oracle_cache = {}


def oracle_pass(proc, n, spec, opdf):
    key = (proc, n, spec)
    if key not in _oracle_cache:
        g = O.vegas_init(IN.DIM[proc], PHYS[proc].n_bins)
        _oracle_cache[key] = O.vegas_pass_obs(proc, PHYS[proc], opdf, g, n, *spec, iteration=0)
    return _oracle_cache[key]


def ctx_for(proc, prec, pdf_grid):
    from paper_2105_10529_gb300.api import Context
    return Context(PHYS[proc], pdf_grid, precision=prec)


def check_bins(gpu, ref, tol):
    scale = np.abs(ref).sum()
    assert np.all(np.abs(gpu - ref) <= tol * np.abs(ref) + 1e-14 * scale), np.max(np.abs(gpu - ref) / (np.abs(ref) + 1e-300))


CASES = [(p, prec) for p in (IN.EE_MUMU, IN.GG_TT, IN.UU_TT, IN.UG_TTU, IN.GG_TTG) for prec in (0, 1)]
CASES += [(IN.GG_TTGG, 0), (IN.GG_TTGG, 1)]


@pytest.mark.parametrize("proc,prec", CASES)
def test_observable_one_pass_matches_oracle(proc, prec, pdf_grid, opdf):
    """One iteration at the uniform grid is one pass over events 0..n-1 of
    Philox iteration 0: the histogram and its per-bin errors against the
    oracle's pass over the same events."""
    n = N_OBS.get(proc, 2001 if prec == 0 else 40011)
    spec = SPEC.get(proc, DEFAULT_SPEC)
    ctx = ctx_for(proc, prec, pdf_grid)
    ctx.set_observable(*spec)
    r = ctx.integrate(proc, PHYS[proc].sqrt_s, n, 1)
    h, e = ctx.observable()
    ctx.close()
    ref = oracle_pass(proc, n, spec, opdf)
    I, S2 = ref["obs"][:, 0], ref["obs"][:, 1]
    check_bins(h, I, TOL[prec])
    var = (n * S2 - I * I) / (n - 1)
    check_bins(e, np.sqrt(np.maximum(var, 0.0)), max(TOL[prec], 1e-9))
    assert h.sum() == pytest.approx(r["sigma"], rel=1e-12)
    assert (h > 0).sum() >= 4                    # the events spread over several bins


def test_observable_iterations_match_oracle(pdf_grid, opdf):
    """Three refined iterations (FP64): every iteration's bins and the
    combination with the integral's inverse-variance weights."""
    proc, n, n_iter, spec = IN.GG_TT, 20000, 3, (8, 0.0, 400.0)
    ctx = ctx_for(proc, 0, pdf_grid)
    ctx.set_observable(*spec)
    r = ctx.integrate(proc, PHYS[proc].sqrt_s, n, n_iter)
    h, e, it = ctx.observable(n_iter)
    ctx.close()
    ref = O.integrate_obs(proc, PHYS[proc], opdf, n, n_iter, *spec)
    assert r["sigma"] == pytest.approx(ref["sigma"], rel=1e-10)
    assert np.allclose(it, ref["per_iter"], rtol=1e-9, atol=1e-12 * ref["sigma"])
    assert np.allclose(h, ref["hist"], rtol=1e-9, atol=0.0)
    assert np.allclose(e, ref["err"], rtol=1e-8, atol=0.0)
    assert h.sum() == pytest.approx(r["sigma"], rel=1e-12)


def test_observable_leaves_the_integral_unchanged(pdf_grid):
    """Filling the histogram changes no weight: the pass counts are identical
    with and without it, and sigma and its error agree to the last bits (the
    histogram's shared memory may change how many CTAs fit, and with them the
    grouping of the partial sums)."""
    for proc, prec, n in ((IN.GG_TT, 1, 100003), (IN.GG_TTGG, 1, 50021), (IN.GG_TTG, 0, 30011)):
        ctx = ctx_for(proc, prec, pdf_grid)
        a = ctx.integrate(proc, PHYS[proc].sqrt_s, n, 2)
        ctx.set_observable(20, 0.0, 600.0)
        b = ctx.integrate(proc, PHYS[proc].sqrt_s, n, 2)
        h, _ = ctx.observable()
        ctx.set_observable(0)
        c = ctx.integrate(proc, PHYS[proc].sqrt_s, n, 2)
        ctx.close()
        assert a["n_pass"] == b["n_pass"] == c["n_pass"], proc
        assert a["sigma"] == c["sigma"] and a["error"] == c["error"], proc
        assert b["sigma"] == pytest.approx(a["sigma"], rel=1e-12), proc
        assert b["error"] == pytest.approx(a["error"], rel=1e-9), proc
        assert h.sum() == pytest.approx(b["sigma"], rel=1e-12)


def test_observable_heavy_schedules_agree(pdf_grid):
    """g g -> t tbar g g mixed: the barrier schedule, the tensor-core colour sum,
    the helicity split and the warp-per-event schedules (diagrams, and the
    helicity-recycled recursion) fill the same histogram up to FP32 rounding."""
    proc, n = IN.GG_TTGG, 60013
    ctx = ctx_for(proc, 1, pdf_grid)
    ctx.set_observable(16, 0.0, 480.0)
    out = []
    for sched, hs in ((1, 1), (2, 1), (1, 2), (2, 2), (3, 1), (4, 1)):
        ctx.set_schedule(sched)
        ctx.set_helicity_split(hs)
        r = ctx.integrate(proc, PHYS[proc].sqrt_s, n, 1)
        h, _ = ctx.observable()
        assert h.sum() == pytest.approx(r["sigma"], rel=1e-12)
        out.append(h)
    ctx.device_status()
    ctx.close()
    for h in out[1:5]:
        assert np.allclose(h, out[0], rtol=1e-6, atol=1e-12 * out[0].sum())
    # the recursion is a different FP32 evaluation: within 2e-5 (two 1e-5 per-event bounds)
    assert np.allclose(out[5], out[0], rtol=2e-5, atol=1e-12 * out[0].sum())


def test_observable_arguments(pdf_grid):
    from paper_2105_10529_gb300._lib import MfError
    proc = IN.GG_TT
    ctx = ctx_for(proc, 1, pdf_grid)
    with pytest.raises(MfError):
        ctx.observable()                      # nothing filled yet
    for bad in ((101, 0.0, 100.0), (-1, 0.0, 100.0), (10, 5.0, 5.0), (10, 0.0, float("inf"))):
        with pytest.raises(MfError):
            ctx.set_observable(*bad)
    ctx.set_observable(4, 0.0, 100.0)
    with pytest.raises(MfError):
        ctx.observable()                      # enabled, but no integration since
    ctx.integrate(proc, PHYS[proc].sqrt_s, 5000, 1)
    h, e = ctx.observable()
    assert h.shape == (6,) and e.shape == (6,)
    ctx.set_observable(0)
    with pytest.raises(MfError):
        ctx.observable()
    ctx.close()

"""Helicity-recycled schedule of the g g -> t tbar g g integrand (schedule 4):
one warp per event builds the colour-ordered partial amplitudes of the 32
configurations of the parity-halved helicity sum from currents that are each
evaluated once per combination of the helicities they depend on (Sec. 2.2's
helicity loop re-associated; Berends-Giele recursion with a closure in the
middle of the top line), then the colour sum on the tensor cores.  It is a
different FP32 evaluation of the same |M|^2, so events agree with the FP64
oracle within the mixed-precision bound (1e-5 per event), and the pass sums
with the diagram schedule (3) to the same rounding."""
import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from tests.gpu_common import PHYS, check_events_against_oracle, oracle_events, random_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROC = IN.GG_TTGG
# two mixed-precision evaluations, each within 1e-5 of the exact per-event value:
# entries of sum w within 2e-5 of each other, entries of sums of w^2 within 4e-5
TOL_W, TOL_W2 = 2e-5, 4e-5


@pytest.fixture(scope="module")
def pdf_grid():
    return IN.make_pdf_grid()


@pytest.fixture(scope="module")
def opdf(pdf_grid):
    return O.Pdf(pdf_grid)


def ctx_for(pdf_grid, phys=None):
    from paper_2105_10529_gb300.api import Context
    return Context(phys or PHYS[PROC], pdf_grid, precision=1)


def assert_sums_close(a, b):
    """Pass sums [sum w, sum w^2, per-bin sums of w^2]: within TOL_W / TOL_W2."""
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    assert abs(a[0] - b[0]) <= TOL_W * abs(a[0]) + 1e-300, (a[0], b[0])
    d = np.abs(a[1:] - b[1:])
    assert np.all(d <= TOL_W2 * np.abs(a[1:]) + 1e-300), (np.argmax(d / (np.abs(a[1:]) + 1e-300)),)


@pytest.mark.parametrize("n", [1, 9, 1001])
def test_events_match_oracle(n, pdf_grid, opdf):
    """A single event, fewer events than warps, a partial last batch in every
    CTA: event by event the bins bit-exact, the masks exact away from a cut
    threshold, |M|^2 and w within 1e-5 of the oracle; the sum of weights
    within 1e-5 of the oracle's; the pass without outputs equal to the pass
    with them bit for bit (one kernel), and within rounding of schedule 3."""
    phys = PHYS[PROC]
    g = random_grid(IN.DIM[PROC], seed=71)
    grid = torch.tensor(g, device="cuda")
    ctx = ctx_for(pdf_grid)
    ctx.set_schedule(4)
    s4, ev = ctx.vegas_pass(PROC, phys.sqrt_s, grid, n, iteration=5, want_events=True,
                            fields=("bins", "mask", "w", "me2"))
    s4n, _ = ctx.vegas_pass(PROC, phys.sqrt_s, grid, n, iteration=5)
    ctx.device_status()
    assert torch.equal(s4, s4n)
    ref = check_events_against_oracle(PROC, phys, opdf, g, ev, 5, 1, what=f"schedule 4, n={n}")
    ref_sum = float(np.sum(ref["w"])) / n
    if ref_sum == 0.0:
        assert float(s4[0]) == 0.0
    else:
        assert float(s4[0]) == pytest.approx(ref_sum, rel=1e-5)
    ctx.set_schedule(3)
    s3, _ = ctx.vegas_pass(PROC, phys.sqrt_s, grid, n, iteration=5)
    assert_sums_close(s3, s4)
    ctx.close()


def test_full_batches_and_event_offset(pdf_grid, opdf):
    """Every CTA through full 256-event batches and a partial one, at an event
    offset beyond 2^32: pass sums within rounding of schedule 3, and 64 events
    spread over the pass against the oracle one by one."""
    phys = PHYS[PROC]
    g = random_grid(IN.DIM[PROC], seed=72)
    grid = torch.tensor(g, device="cuda")
    ctx = ctx_for(pdf_grid)
    n, off = 120_001, (1 << 32) - 5000
    ctx.set_schedule(3)
    s3, _ = ctx.vegas_pass(PROC, phys.sqrt_s, grid, n, ev_offset=off, iteration=7)
    ctx.set_schedule(4)
    s4, ev = ctx.vegas_pass(PROC, phys.sqrt_s, grid, n, ev_offset=off, iteration=7, want_events=True,
                            fields=("bins", "mask", "w", "me2"))
    ctx.device_status()
    assert float(s4[0]) > 0.0
    assert_sums_close(s3, s4)
    rng = np.random.default_rng(73)
    idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 62)]))
    check_events_against_oracle(PROC, phys, opdf, g, ev, 7, 1, first=off, events=idx, what="schedule 4, offset")
    ctx.close()


def test_full_size_pass_sampled(pdf_grid, opdf):
    """The benchmark's pass (4e6 events of its physics, uniform grid) under
    schedule 4 with per-event outputs: 150 seeded events and the first and last
    against the oracle one by one (bins exact, w and |M|^2 within 1e-5), and
    the sums within rounding of schedule 3 on the same events."""
    phys = IN.Physics(seed=3)
    dim = IN.DIM[PROC]
    g = np.tile(np.linspace(0.0, 1.0, phys.n_bins + 1), (dim, 1))
    grid = torch.tensor(g, device="cuda")
    ctx = ctx_for(pdf_grid, phys)
    n = 4_000_000
    ctx.set_schedule(4)
    s4, ev = ctx.vegas_pass(PROC, phys.sqrt_s, grid, n, iteration=3, want_events=True,
                            fields=("bins", "mask", "w", "me2"))
    ctx.set_schedule(3)
    s3, _ = ctx.vegas_pass(PROC, phys.sqrt_s, grid, n, iteration=3)
    ctx.device_status()
    assert_sums_close(s3, s4)
    rng = np.random.default_rng(74)
    idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 150)]))
    check_events_against_oracle(PROC, phys, opdf, g, ev, 3, 1, events=idx, what="schedule 4, full size")
    ctx.close()


def test_integrate_and_observable(pdf_grid):
    """Iterated VEGAS with the p_T histogram on: sigma, the pass count and
    every histogram bin within rounding of schedule 3 (the refined grids follow
    the sums, so the later iterations see the same events)."""
    phys = PHYS[PROC]
    ctx = ctx_for(pdf_grid)
    ctx.set_observable(20, 0.0, 800.0)
    out = {}
    for sched in (3, 4):
        ctx.set_schedule(sched)
        r = ctx.integrate(PROC, phys.sqrt_s, 30000, 3)
        ctx.device_status()
        out[sched] = (r, ctx.observable())
    (r3, o3), (r4, o4) = out[3], out[4]
    assert r4["sigma"] == pytest.approx(r3["sigma"], rel=TOL_W)
    assert r4["n_pass"] == r3["n_pass"] and r4["n_nan"] == r3["n_nan"] == 0
    h3, h4 = np.asarray(o3[0]), np.asarray(o4[0])
    assert np.all(np.abs(h4 - h3) <= TOL_W * np.abs(h3) + 1e-12 * abs(r3["sigma"]))
    ctx.close()


def test_other_processes_and_precisions_fall_back(pdf_grid):
    """Schedule 4 applies to g g -> t tbar g g in mixed precision; other processes
    run it as schedule 3 (bit for bit), and 5 is rejected."""
    phys = PHYS[PROC]
    ctx = ctx_for(pdf_grid)
    p = IN.GG_TTG
    g3 = torch.tensor(random_grid(IN.DIM[p], seed=75), device="cuda")
    ctx.set_schedule(3)
    t3, _ = ctx.vegas_pass(p, phys.sqrt_s, g3, 2000, iteration=1)
    ctx.set_schedule(4)
    t4, _ = ctx.vegas_pass(p, phys.sqrt_s, g3, 2000, iteration=1)
    assert torch.equal(t3, t4)
    ctx.device_status()
    from paper_2105_10529_gb300._lib import MfError
    with pytest.raises(MfError):
        ctx.set_schedule(5)
    ctx.close()

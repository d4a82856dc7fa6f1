"""Warp-per-event schedule of the g g -> t tbar g g integrand (schedule 3):
one warp per event, one lane per helicity of the parity-halved sum (Sec. 2.2),
the colour sum on the tensor cores.  It evaluates the same amplitudes as
schedule 2 and adds the 32 helicities in another order, so every pass sum
agrees with schedule 2 to FP32 rounding, the event counts exactly, and the
sum of weights with the FP64 oracle within the mixed-precision bound."""
import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from tests.gpu_common import PHYS, check_events_against_oracle, oracle_events, random_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROC = IN.GG_TTGG


@pytest.fixture(scope="module")
def pdf_grid():
    return IN.make_pdf_grid()


@pytest.fixture(scope="module")
def opdf(pdf_grid):
    return O.Pdf(pdf_grid)


def ctx_for(pdf_grid, phys=None):
    from paper_2105_10529_gb300.api import Context
    return Context(phys or PHYS[PROC], pdf_grid, precision=1)


def pass_pair(ctx, phys, grid, n, iteration, offset=0):
    ctx.set_schedule(2)
    a, _ = ctx.vegas_pass(PROC, phys.sqrt_s, grid, n, ev_offset=offset, iteration=iteration)
    ctx.set_schedule(3)
    b, _ = ctx.vegas_pass(PROC, phys.sqrt_s, grid, n, ev_offset=offset, iteration=iteration)
    ctx.device_status()
    return a, b


@pytest.mark.parametrize("n", [1, 9, 1001])
def test_pass_matches_schedule_2_and_oracle(n, pdf_grid, opdf):
    """Small and ragged passes (a single event, fewer events than warps, a
    partial last batch in every CTA): every entry of the pass sums within
    1e-6 of schedule 2, the sum of weights within 1e-5 of the oracle's, and
    event by event (the same kernel writing its per-event outputs) the
    bins bit-exact and |M|^2 and w within 1e-5 of the oracle."""
    phys = PHYS[PROC]
    g = random_grid(IN.DIM[PROC], seed=61)
    grid = torch.tensor(g, device="cuda")
    ctx = ctx_for(pdf_grid)
    a, b = pass_pair(ctx, phys, grid, n, iteration=4)
    assert torch.all((a - b).abs() <= 1e-6 * a.abs() + 1e-300)
    ref = oracle_events(PROC, phys, opdf, g, n, iteration=4)
    ref_sum = float(np.sum(ref["w"])) / n
    if ref_sum == 0.0:
        assert float(b[0]) == 0.0
    else:
        assert float(b[0]) == pytest.approx(ref_sum, rel=1e-5)
    # schedule 3 with per-event outputs: the same kernel, so the same sums bit for bit
    ctx.set_schedule(3)
    c, ev = ctx.vegas_pass(PROC, phys.sqrt_s, grid, n, iteration=4, want_events=True,
                           fields=("bins", "mask", "w", "me2"))
    ctx.device_status()
    assert torch.equal(c, b)
    check_events_against_oracle(PROC, phys, opdf, g, ev, 4, 1, what=f"schedule 3, n={n}")
    ctx.close()


def test_full_batches_and_event_offset(pdf_grid):
    """Enough events that every CTA evaluates full 256-event batches and a
    partial one, at an event offset beyond 2^32: pass sums within 1e-6 of
    schedule 2 entry by entry."""
    phys = PHYS[PROC]
    grid = torch.tensor(random_grid(IN.DIM[PROC], seed=62), device="cuda")
    ctx = ctx_for(pdf_grid)
    a, b = pass_pair(ctx, phys, grid, 120_001, iteration=7, offset=(1 << 32) - 5000)
    assert float(a[0]) > 0.0
    assert torch.all((a - b).abs() <= 1e-6 * a.abs() + 1e-300)
    ctx.close()


def test_full_size_pass(pdf_grid):
    """The benchmark's pass (4e6 events, its physics) under both schedules:
    the sums agree to FP32 rounding."""
    phys = IN.Physics(seed=3)
    dim = IN.DIM[PROC]
    grid = torch.linspace(0, 1, phys.n_bins + 1, dtype=torch.float64, device="cuda").repeat(dim, 1).contiguous()
    ctx = ctx_for(pdf_grid, phys)
    a, b = pass_pair(ctx, phys, grid, 4_000_000, iteration=3)
    assert torch.all((a - b).abs() <= 1e-6 * a.abs() + 1e-300)
    ctx.close()


def test_integrate_and_observable(pdf_grid):
    """Iterated VEGAS with the p_T histogram on: sigma, the pass count and
    every histogram bin agree with schedule 2 to rounding."""
    phys = PHYS[PROC]
    ctx = ctx_for(pdf_grid)
    ctx.set_observable(20, 0.0, 800.0)
    out = {}
    for sched in (2, 3):
        ctx.set_schedule(sched)
        r = ctx.integrate(PROC, phys.sqrt_s, 30000, 3)
        ctx.device_status()
        out[sched] = (r, ctx.observable())
    (r2, o2), (r3, o3) = out[2], out[3]
    assert r3["sigma"] == pytest.approx(r2["sigma"], rel=1e-6)
    assert r3["n_pass"] == r2["n_pass"] and r3["n_nan"] == r2["n_nan"] == 0
    h2, h3 = np.asarray(o2[0]), np.asarray(o3[0])
    assert np.all(np.abs(h3 - h2) <= 1e-6 * np.abs(h2) + 1e-12 * abs(r2["sigma"]))
    ctx.close()


def test_per_event_outputs_and_other_processes_fall_back(pdf_grid):
    """Per-event outputs run schedule 3 itself (|M|^2 within FP32 rounding of
    schedule 2, the sums equal to those of the pass without outputs); the
    helicity split and processes without the tensor-core colour sum run
    schedule 3 as schedule 2; 5 is rejected."""
    phys = PHYS[PROC]
    grid = torch.tensor(random_grid(IN.DIM[PROC], seed=63), device="cuda")
    ctx = ctx_for(pdf_grid)
    ctx.set_schedule(2)
    _, e2 = ctx.vegas_pass(PROC, phys.sqrt_s, grid, 300, iteration=1, want_events=True, fields=("me2",))
    ctx.set_schedule(3)
    s3, e3 = ctx.vegas_pass(PROC, phys.sqrt_s, grid, 300, iteration=1, want_events=True, fields=("me2",))
    s3n, _ = ctx.vegas_pass(PROC, phys.sqrt_s, grid, 300, iteration=1)
    assert torch.equal(s3, s3n)
    m2, m3 = e2["me2"].cpu().numpy(), e3["me2"].cpu().numpy()
    assert np.array_equal(m2 == 0, m3 == 0)
    nz = m2 != 0
    assert np.all(np.abs(m3[nz] - m2[nz]) <= 1e-6 * np.abs(m2[nz]))
    ctx.set_helicity_split(2)
    s3, _ = ctx.vegas_pass(PROC, phys.sqrt_s, grid, 700, iteration=1)
    ctx.set_schedule(2)
    s2, _ = ctx.vegas_pass(PROC, phys.sqrt_s, grid, 700, iteration=1)
    assert torch.equal(s2, s3)
    ctx.set_helicity_split(1)
    p = IN.GG_TTG
    g3 = torch.tensor(random_grid(IN.DIM[p], seed=64), device="cuda")
    t2, _ = ctx.vegas_pass(p, phys.sqrt_s, g3, 2000, iteration=1)
    ctx.set_schedule(3)
    t3, _ = ctx.vegas_pass(p, phys.sqrt_s, g3, 2000, iteration=1)
    assert torch.equal(t2, t3)
    ctx.device_status()
    from paper_2105_10529_gb300._lib import MfError
    with pytest.raises(MfError):
        ctx.set_schedule(5)
    ctx.close()

"""g g -> t tbar g g g (row f2: the multi-leg process; the paper's Sec. 4
names multi-leg processes as the next step): the warp-level Berends-Giele
matrix element and the integrand around it, through the C ABI, against the
FP64 oracle (five-gluon Berends-Giele with Dirac spinors and a brute-force
colour matrix).  Bit-exact random numbers, bins and mapped points; masks
bit-exact away from a threshold; |M|^2 and weights within the per-event
bounds (FP64) and 1e-5 (mixed)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from tests.gpu_common import (EPS, assert_fp_parity, check_events_against_oracle, fp64_event_bounds,
                              me_condition, oracle_events, random_grid, rel_err)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROC = IN.GG_TTGGG
PHYS = IN.Physics(seed=6)


@pytest.fixture(scope="module")
def pdf_grid():
    return IN.make_pdf_grid()


@pytest.fixture(scope="module")
def opdf(pdf_grid):
    return O.Pdf(pdf_grid)


def ctx_for(prec, pdf_grid, phys=PHYS):
    from paper_2105_10529_gb300.api import Context
    return Context(phys, pdf_grid, precision=prec)


def points(n_per_shat, seed):
    rng = np.random.default_rng(seed)
    moms = []
    for shat_tev2 in (0.5, 1.0, 3.0, 13.0):
        rs = math.sqrt(shat_tev2) * 1000.0
        for _ in range(n_per_shat):
            pf, _ = O.rambo(5, rs, [PHYS.mt, PHYS.mt, 0.0, 0.0, 0.0], rng.random(20))
            moms.append(np.vstack([[[rs / 2, 0, 0, rs / 2], [rs / 2, 0, 0, -rs / 2]], pf]))
    return np.array(moms)


def test_process_info():
    from paper_2105_10529_gb300.api import process_info
    assert process_info(PROC) == (7, 22)


@pytest.mark.parametrize("prec", [0, 1])
def test_evaluate_parity(prec, pdf_grid):
    moms = points(6, 600)
    refs = np.array([O.me2(PROC, PHYS, p) for p in moms])
    ctx = ctx_for(prec, pdf_grid)
    out = ctx.evaluate(PROC, torch.tensor(moms, device="cuda")).cpu().numpy()
    bound = np.array([max(1e-12, 64 * EPS * me_condition(PROC, PHYS, p)) for p in moms])
    assert_fp_parity(rel_err(out, refs), prec, "evaluate", bound if prec == 0 else None)
    # an empty batch is a no-op
    ctx.evaluate(PROC, torch.zeros((0, 7, 4), dtype=torch.float64, device="cuda"))
    ctx.close()


@pytest.mark.parametrize("prec,n", [(0, 97), (1, 301)])
def test_event_parity(prec, n, pdf_grid, opdf):
    """A pass over several CTAs' batches and a ragged tail: uniforms, mapped
    points and bins bit for bit, masks, and w and |M|^2 event by event."""
    dim = IN.DIM[PROC]
    grid = random_grid(dim, seed=66)
    ctx = ctx_for(prec, pdf_grid)
    sums, ev = ctx.vegas_pass(PROC, PHYS.sqrt_s, torch.tensor(grid, device="cuda"), n, iteration=2,
                              want_events=True)
    ctx.device_status()
    ref = oracle_events(PROC, PHYS, opdf, grid, n, iteration=2)
    assert np.array_equal(ev["u"].cpu().numpy(), ref["u"])
    assert np.array_equal(ev["x"].cpu().numpy(), ref["x"])
    assert np.array_equal(ev["bins"].cpu().numpy(), ref["bins"])
    assert int(ref["mask"].sum()) > n // 4
    check_events_against_oracle(PROC, PHYS, opdf, grid, {k: ev[k] for k in ("bins", "mask", "w", "me2")}, 2, prec,
                                what=f"gg_ttggg prec {prec}")
    s = sums.cpu().numpy()
    sw = ref["w"].sum() / n
    assert abs(s[0] - sw) <= (1e-11 if prec == 0 else 1e-5) * abs(sw)
    # the same kernel without outputs: the same sums
    plain, _ = ctx.vegas_pass(PROC, PHYS.sqrt_s, torch.tensor(grid, device="cuda"), n, iteration=2)
    assert torch.equal(plain, sums)
    ctx.close()


def test_helicity_profile():
    """Rows add up to evaluate's |M|^2; parity mirrors agree helicity by helicity (FP64)."""
    moms = points(3, 601)
    ctx = ctx_for(0, IN.make_pdf_grid())
    mt = torch.tensor(moms, device="cuda")
    prof = ctx.helicity_profile(PROC, mt).cpu().numpy()
    me = ctx.evaluate(PROC, mt).cpu().numpy()
    ctx.close()
    assert prof.shape == (len(moms), 128)
    assert np.all(rel_err(prof.sum(1), me) < 1e-13)
    mirror = prof[:, [ih ^ 127 for ih in range(128)]]
    assert np.all(np.abs(prof - mirror) <= 1e-12 * prof.max(1, keepdims=True))


def test_integrate_matches_oracle(pdf_grid, opdf):
    """Two refined iterations in FP64: the GPU and the oracle run the same
    algorithm on the same random numbers, so sigma and the grids agree far
    below the Monte Carlo error."""
    n = 1200
    ctx = ctx_for(0, pdf_grid)
    r = ctx.integrate(PROC, PHYS.sqrt_s, n, 2, want_grid=True)
    ctx.close()
    ref = O.integrate(PROC, PHYS, opdf, n, 2)
    assert abs(r["sigma"] - ref["sigma"]) < 1e-9 * abs(ref["sigma"])
    assert np.abs(r["grid"] - ref["grid"]).max() < 1e-9
    assert r["n_pass"] == ref["n_pass"]


def test_full_size_pass_sampled_against_oracle(pdf_grid, opdf):
    """The benchmark leg's pass size (1e6 events, mixed precision, one CTA per
    SM): a seeded sample of events, the first and the last, recomputed one by
    one by the oracle; the pass sums equal the sums of the per-event weights."""
    n = 1_000_000
    grid = random_grid(IN.DIM[PROC], seed=67)
    ctx = ctx_for(1, pdf_grid)
    sums, ev = ctx.vegas_pass(PROC, PHYS.sqrt_s, torch.tensor(grid, device="cuda"), n, iteration=4,
                              want_events=True, fields=("bins", "w", "mask", "me2"))
    ctx.device_status()
    w = ev["w"].cpu().numpy()
    assert abs(float(sums[0]) - w.sum() / n) <= 1e-12 * abs(w.sum() / n)
    rng = np.random.default_rng(2025)
    sample = np.concatenate([[0, n - 1], rng.choice(n, 62, replace=False)])
    check_events_against_oracle(PROC, PHYS, opdf, grid, ev, 4, 1, events=sample, what="gg_ttggg full size")
    ctx.close()


def test_not_in_batches(pdf_grid):
    from paper_2105_10529_gb300._lib import MfError
    ctx = ctx_for(1, pdf_grid)
    with pytest.raises(MfError):
        ctx.integrate_batch([IN.GG_TT, PROC], [1000, 1000], PHYS.sqrt_s, 1)
    ctx.close()

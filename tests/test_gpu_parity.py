"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Bit-exact for random streams, VEGAS bins and mapped
points and cut masks (away from a threshold); per-event weights within 1e-12
(FP64 path) and 1e-5 (mixed path) relative."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from tests.gpu_common import (EPS, PHYS, assert_fp_parity, check_events_against_oracle, cut_margin,
                              fp64_event_bounds, me_condition, oracle_events, rambo_gamma, random_grid, rel_err)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROCS = [IN.EE_MUMU, IN.GG_TT, IN.GG_TTG, IN.GG_TTGG, IN.UU_TT, IN.UG_TTU]
N_SMALL = {IN.EE_MUMU: 4099, IN.GG_TT: 3001, IN.GG_TTG: 1501, IN.GG_TTGG: 301, IN.UU_TT: 3001, IN.UG_TTU: 1201}
TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def pdf_grid():
    return IN.make_pdf_grid()


@pytest.fixture(scope="module")
def opdf(pdf_grid):
    return O.Pdf(pdf_grid)


def ctx_for(proc, prec, pdf_grid):
    from paper_2105_10529_gb300.api import Context
    return Context(PHYS[proc], pdf_grid, precision=prec)


@pytest.mark.parametrize("proc", PROCS)
@pytest.mark.parametrize("prec", [0, 1])
def test_event_parity(proc, prec, pdf_grid, opdf):
    phys = PHYS[proc]
    dim = IN.DIM[proc]
    n = N_SMALL[proc]
    grid = random_grid(dim, seed=proc)
    ctx = ctx_for(proc, prec, pdf_grid)
    g = torch.tensor(grid, device="cuda")
    it = 3
    sums, ev = ctx.vegas_pass(proc, phys.sqrt_s, g, n, ev_offset=0, iteration=it, want_events=True)
    torch.cuda.synchronize()
    ref = oracle_events(proc, phys, opdf, grid, n, iteration=it)
    u = ev["u"].cpu().numpy(); x = ev["x"].cpu().numpy(); b = ev["bins"].cpu().numpy()
    # random stream, bins and mapped points: bit-exact
    assert np.array_equal(u, ref["u"])
    assert np.array_equal(b, ref["bins"])
    assert np.array_equal(x, ref["x"])
    # cut masks: bit-exact except for events within rounding of a threshold
    mk = ev["mask"].cpu().numpy().astype(int)
    flips = np.nonzero(mk != ref["mask"])[0]
    for i in flips:
        assert cut_margin(proc, phys, ref["plab"][i]) < 1e-9, f"mask flip far from threshold at event {i}"
    same = mk == ref["mask"]
    b_me, b_w = fp64_event_bounds(proc, phys, opdf, ref, ev["momenta"].cpu().numpy()) if prec == 0 else (None, None)
    w = ev["w"].cpu().numpy()
    assert_fp_parity(rel_err(w[same], ref["w"][same]), prec, "w", b_w[same] if prec == 0 else None)
    me = ev["me2"].cpu().numpy()
    assert_fp_parity(rel_err(me[same], ref["me2"][same]), prec, "me2", b_me[same] if prec == 0 else None)
    # momenta in the partonic frame, per event relative to the event's largest
    # component.  RAMBO's conformal map scales the massless momenta by
    # sqrt(shat)/M and boosts them with gamma = Q0/M (Q the sum of the isotropic
    # momenta, M its mass), so a relative rounding difference eps of the inputs
    # (libm against CUDA log / sincospi) reaches the outputs as about
    # gamma^2 eps; the bound is 4500 eps or 8 gamma^2 eps, whichever is larger.
    # eps is the kinematics' own: FP64's 2^-52 on the FP64 path, and on the mixed
    # path, whose kinematics run in double-float (two floats, 48 bits), 2^-47.
    eps = np.finfo(float).eps if prec == 0 or proc == IN.EE_MUMU else 2.0 ** -47
    floor = 4500.0 * eps
    pm = ev["momenta"].cpu().numpy()
    scale = np.abs(ref["p"]).reshape(n, -1).max(axis=1)
    dev = np.abs(pm - ref["p"]).reshape(n, -1).max(axis=1) / scale
    gam = np.ones(n) if proc == IN.EE_MUMU else rambo_gamma(ref["x"], IN.N_EXT[proc] - 2)
    bound = np.maximum(floor, 8.0 * gam ** 2 * eps)
    assert np.all(dev <= bound), (int(np.argmax(dev / bound)), float(np.max(dev / bound)))
    assert np.mean(dev > floor) <= 5e-3 or int(np.sum(dev > floor)) <= 1
    # pass sums (w includes 1/n)
    s = sums.cpu().numpy()
    sw = ref["w"].sum() / n
    assert abs(s[0] - sw) <= (1e-11 if prec == 0 else 1e-5) * abs(sw) + 1e-300
    ctx.close()


@pytest.mark.parametrize("proc", PROCS)
def test_fp64_me_at_identical_momenta(proc, pdf_grid, opdf):
    """The FP64 tail separated from the kinematics: the oracle's |M|^2 evaluated
    at the GPU's own per-event momenta agrees with the GPU's |M|^2 event by
    event to 1e-12, or to 64 eps times the event's condition number where a
    final particle runs along a beam (2 E^2 / (m^2 + pT^2), the cancellation in
    p_beam . p_i); the GPU's momenta are on their mass shells and conserve
    momentum to rounding (the RAMBO map's gamma^2 eps for the massless ones)."""
    phys = PHYS[proc]
    n = N_SMALL[proc]
    grid = random_grid(IN.DIM[proc], seed=proc)
    ctx = ctx_for(proc, 0, pdf_grid)
    _, ev = ctx.vegas_pass(proc, phys.sqrt_s, torch.tensor(grid, device="cuda"), n, iteration=3, want_events=True,
                           fields=("x", "mask", "me2", "momenta"))
    ctx.close()
    mk = ev["mask"].cpu().numpy().astype(bool)
    pm = ev["momenta"].cpu().numpy()[mk]
    me = ev["me2"].cpu().numpy()[mk]
    at = np.array([O.me2(proc, phys, p) for p in pm])
    bound = np.array([max(1e-12, 64 * EPS * me_condition(proc, phys, p)) for p in pm])
    err = rel_err(me, at)
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, [(int(i), float(err[i]), float(bound[i])) for i in bad[:5]]
    assert np.median(err) < 1e-14
    # mass shells (relative to E^2) and momentum conservation (relative to sqrt(shat))
    n_ext = IN.N_EXT[proc]
    masses = np.array([0.0, 0.0] + ([0.0, 0.0] if proc == IN.EE_MUMU else [phys.mt, phys.mt]) + [0.0] * (n_ext - 4))
    p2 = pm[..., 0] ** 2 - (pm[..., 1:] ** 2).sum(-1)
    shell = np.abs(p2 - masses ** 2) / pm[..., 0] ** 2
    gam = np.ones(len(pm)) if proc == IN.EE_MUMU else rambo_gamma(ev["x"].cpu().numpy()[mk], n_ext - 2)
    assert np.all(shell.max(axis=1) <= np.maximum(1e-14, 16 * gam ** 2 * EPS)), float(shell.max())
    if proc in (IN.GG_TT, IN.UU_TT):
        assert shell.max() < 1e-14        # the 2 -> 2 pair is built on shell, back to back
    cons = np.abs(pm[:, :2].sum(1) - pm[:, 2:].sum(1)).max(axis=1) / (2 * pm[:, 0, 0])
    assert np.all(cons <= np.maximum(1e-14, 16 * gam ** 2 * EPS)), float(cons.max())


@pytest.mark.parametrize("proc", PROCS)
@pytest.mark.parametrize("prec", [0, 1])
def test_evaluate_parity(proc, prec, pdf_grid):
    phys = PHYS[proc]
    rng = np.random.default_rng(100 + proc)
    n_ext = IN.N_EXT[proc]
    nf = n_ext - 2
    masses = {IN.EE_MUMU: [0.0, 0.0]}.get(proc, [phys.mt, phys.mt] + [0.0] * (nf - 2))
    moms, refs = [], []
    for shat_tev2 in (0.5, 1.0, 3.0, 13.0):
        rs = math.sqrt(shat_tev2) * 1000.0 if proc != IN.EE_MUMU else 91.19 * shat_tev2
        for _ in range(8):
            pf, _ = O.rambo(nf, rs, masses, rng.random(4 * nf))
            p = np.vstack([[[rs / 2, 0, 0, rs / 2], [rs / 2, 0, 0, -rs / 2]], pf])
            moms.append(p)
            refs.append(O.me2(proc, phys, p))
    ctx = ctx_for(proc, prec, pdf_grid)
    out = ctx.evaluate(proc, torch.tensor(np.array(moms), device="cuda")).cpu().numpy()
    bound = np.array([max(1e-12, 64 * EPS * me_condition(proc, phys, p)) for p in moms])
    assert_fp_parity(rel_err(out, refs), prec, "evaluate", bound if prec == 0 else None)
    # empty batch is a no-op
    ctx.evaluate(proc, torch.zeros((0, n_ext, 4), dtype=torch.float64, device="cuda"))
    ctx.close()


def test_ragged_offsets_and_single_event(pdf_grid, opdf):
    proc = IN.GG_TT
    phys = PHYS[proc]
    grid = random_grid(IN.DIM[proc], seed=7)
    ctx = ctx_for(proc, 0, pdf_grid)
    g = torch.tensor(grid, device="cuda")
    for n, off in [(1, 0), (1, 123456789), (37, 5), (1025, 99)]:
        sums, ev = ctx.vegas_pass(proc, phys.sqrt_s, g, n, ev_offset=off, iteration=1, want_events=True,
                                  fields=("u", "w"))
        ref = oracle_events(proc, phys, opdf, grid, n, iteration=1, first=off)
        assert np.array_equal(ev["u"].cpu().numpy(), ref["u"])
        assert_fp_parity(rel_err(ev["w"].cpu().numpy(), ref["w"]), 0, "w", fp64_event_bounds(proc, phys, opdf, ref)[1])
        assert abs(sums[0].item() - ref["w"].sum() / n) <= 1e-11 * abs(ref["w"].sum() / n)
    ctx.close()


def test_frozen_masks(pdf_grid, opdf):
    proc = IN.GG_TTG
    phys = PHYS[proc]
    grid = random_grid(IN.DIM[proc], seed=8)
    ctx = ctx_for(proc, 0, pdf_grid)
    g = torch.tensor(grid, device="cuda")
    n = 500
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    mask[::3] = 1
    sums, ev = ctx.vegas_pass(proc, phys.sqrt_s, g, n, mask_in=mask, want_events=True, fields=("mask", "w"))
    assert np.array_equal(ev["mask"].cpu().numpy(), mask.cpu().numpy())
    w = ev["w"].cpu().numpy()
    assert np.all(w[1::3] == 0) and np.all(w[2::3] == 0)
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_integrate_matches_oracle_ee(prec, pdf_grid, opdf):
    """Same random numbers, same algorithm: GPU and oracle integrals agree far
    below the MC error, and both agree with the closed form within it."""
    proc = IN.EE_MUMU
    phys = PHYS[proc]
    ctx = ctx_for(proc, prec, pdf_grid)
    r = ctx.integrate(proc, phys.sqrt_s, 100_000, 5, want_grid=True)
    ref = O.integrate(proc, phys, opdf, 100_000, 5)
    assert abs(r["sigma"] - ref["sigma"]) < (1e-9 if prec == 0 else 1e-5) * ref["sigma"]
    assert abs(r["error"] / ref["error"] - 1) < (1e-6 if prec == 0 else 1e-3)
    assert np.abs(r["grid"] - ref["grid"]).max() < (1e-9 if prec == 0 else 1e-6)
    from tests.test_oracle_integration import sigma_ee_quadrature
    assert abs(r["sigma"] - sigma_ee_quadrature(phys)) < 3 * r["error"]
    assert r["n_pass"] == 500_000 and r["n_nan"] == 0
    ctx.close()


def test_integrate_matches_oracle_gg_tt(pdf_grid, opdf):
    proc = IN.GG_TT
    phys = PHYS[proc]
    ctx = ctx_for(proc, 0, pdf_grid)
    r = ctx.integrate(proc, phys.sqrt_s, 50_000, 3, want_grid=True)
    ref = O.integrate(proc, phys, opdf, 50_000, 3)
    assert abs(r["sigma"] - ref["sigma"]) < 1e-9 * ref["sigma"]
    assert np.abs(r["grid"] - ref["grid"]).max() < 1e-9
    ctx.close()


def test_bad_arguments(pdf_grid):
    from paper_2105_10529_gb300._lib import MfError
    ctx = ctx_for(IN.GG_TT, 0, pdf_grid)
    g = torch.tensor(random_grid(10), device="cuda")
    with pytest.raises(MfError):
        ctx.integrate(IN.GG_TT, 13000.0, 1, 2)           # n_events < 2
    with pytest.raises(MfError):
        ctx.integrate(IN.GG_TT, 100.0, 1000, 2)          # below threshold
    from paper_2105_10529_gb300.api import Context
    one_flavour = Context(PHYS[IN.GG_TT], IN.make_pdf_grid()[:1], precision=0)
    with pytest.raises(MfError) as e:
        one_flavour.integrate(IN.UU_TT, 13000.0, 1000, 2)   # the grid has no u / ubar
    assert e.value.code == 1
    one_flavour.close()
    with pytest.raises(MfError):
        ctx.vegas_pass(IN.GG_TT, 13000.0, g, 0)
    with pytest.raises(MfError):
        ctx.integrate(17, 13000.0, 1000, 2)
    with pytest.raises(MfError):
        ctx.set_schedule(5)
    ctx.device_status()
    ctx.close()


@pytest.mark.parametrize("proc", [IN.GG_TTG, IN.GG_TTGG])
def test_schedules_give_identical_sums(proc, pdf_grid):
    """The CTA-barrier schedule changes only when warps wait, not what they compute."""
    phys = PHYS[proc]
    grid = torch.tensor(random_grid(IN.DIM[proc], seed=11), device="cuda")
    ctx = ctx_for(proc, 1, pdf_grid)
    n = 3000
    ctx.set_schedule(0)
    a, _ = ctx.vegas_pass(proc, phys.sqrt_s, grid, n, iteration=4)
    ctx.set_schedule(1)
    b, _ = ctx.vegas_pass(proc, phys.sqrt_s, grid, n, iteration=4)
    assert torch.equal(a, b)
    ctx.close()


def test_tensor_core_colour_sum_event_parity(pdf_grid, opdf):
    """Schedule 2 (g g -> t tbar g g colour sum on the tensor cores): every
    event within the mixed-precision bound of the oracle, the same masks and
    bins as schedule 1, and |M|^2 within 1e-6 of schedule 1 (FP32 rounding of
    the two colour-sum orders)."""
    proc = IN.GG_TTGG
    phys = PHYS[proc]
    n = 1001     # several CTAs of 128 events and a ragged last batch
    grid = random_grid(IN.DIM[proc], seed=21)
    g = torch.tensor(grid, device="cuda")
    ctx = ctx_for(proc, 1, pdf_grid)
    ctx.set_schedule(1)
    s1, e1 = ctx.vegas_pass(proc, phys.sqrt_s, g, n, iteration=2, want_events=True)
    ctx.set_schedule(2)
    s2, e2 = ctx.vegas_pass(proc, phys.sqrt_s, g, n, iteration=2, want_events=True)
    ctx.device_status()
    assert torch.equal(e1["mask"], e2["mask"]) and torch.equal(e1["bins"], e2["bins"])
    m1 = e1["me2"].cpu().numpy(); m2 = e2["me2"].cpu().numpy()
    assert rel_err(m2, m1).max() < 1e-6
    ref = oracle_events(proc, phys, opdf, grid, n, iteration=2)
    same = e2["mask"].cpu().numpy().astype(int) == ref["mask"]
    assert_fp_parity(rel_err(m2[same], ref["me2"][same]), 1, "me2 (tensor-core colour sum)")
    w = e2["w"].cpu().numpy()
    assert_fp_parity(rel_err(w[same], ref["w"][same]), 1, "w (tensor-core colour sum)")
    assert abs(float(s2[0]) - float(s1[0])) <= 1e-6 * abs(float(s1[0]))
    ctx.close()


def test_tensor_core_colour_sum_integrate(pdf_grid):
    """Iterated VEGAS with the tensor-core colour sum agrees with schedule 1
    to rounding, and the device reports no expired wait."""
    proc = IN.GG_TTGG
    phys = PHYS[proc]
    ctx = ctx_for(proc, 1, pdf_grid)
    ctx.set_schedule(1)
    r1 = ctx.integrate(proc, phys.sqrt_s, 20000, 2)
    ctx.set_schedule(2)
    r2 = ctx.integrate(proc, phys.sqrt_s, 20000, 2)
    ctx.device_status()
    assert r2["sigma"] == pytest.approx(r1["sigma"], rel=1e-6)
    assert r2["n_pass"] == r1["n_pass"]
    ctx.close()


def test_cuts_argument(pdf_grid):
    """The per-call cuts of mf_integrate: the configuration's values give the
    same result as no argument, a looser pT cut a larger cross section, and
    the grad pass honours them too."""
    proc = IN.GG_TTG
    phys = PHYS[proc]
    ctx = ctx_for(proc, 1, pdf_grid)
    a = ctx.integrate(proc, phys.sqrt_s, 20000, 2)
    b = ctx.integrate(proc, phys.sqrt_s, 20000, 2, cuts=(phys.pt_min, phys.eta_max, phys.dr_min))
    assert a["sigma"] == b["sigma"] and a["n_pass"] == b["n_pass"]
    c = ctx.integrate(proc, phys.sqrt_s, 20000, 2, cuts=(20.0, phys.eta_max, phys.dr_min))
    assert c["n_pass"] > a["n_pass"] and c["sigma"] > a["sigma"]
    d = ctx.integrate(proc, phys.sqrt_s, 20000, 2, cuts=(20.0, 0.0, 0.0))     # no eta cut
    assert d["n_pass"] > c["n_pass"]
    ctx.close()


def test_full_size_pass_sampled_against_oracle(pdf_grid, opdf):
    """The benchmark's workload at full size and in its launch configuration:
    one mixed-precision pass of 4e6 g g -> t tbar g g events under the
    default warp-per-event schedule 3 (one 256-thread CTA per SM), with
    per-event outputs written by that same kernel (its sums equal those of
    the pass without outputs bit for bit); a seeded sample of events, the
    first and the last is recomputed one by one by the oracle, and the pass
    sums equal the sums of the per-event weights."""
    proc = IN.GG_TTGG
    phys = IN.Physics(seed=3)            # the benchmark's physics
    n = 4_000_000
    grid = random_grid(IN.DIM[proc], seed=31)
    from paper_2105_10529_gb300.api import Context
    ctx = Context(phys, pdf_grid, precision=1)
    g = torch.tensor(grid, device="cuda")
    plain, _ = ctx.vegas_pass(proc, phys.sqrt_s, g, n, iteration=5)
    sums, ev = ctx.vegas_pass(proc, phys.sqrt_s, g, n, iteration=5, want_events=True,
                              fields=("bins", "w", "mask", "me2"))
    ctx.device_status()
    assert torch.equal(plain, sums)
    w = ev["w"].cpu().numpy()
    # pass sums from the per-event weights (sum order differs: 1e-12)
    assert abs(float(sums[0]) - w.sum() / n) <= 1e-12 * abs(w.sum() / n)
    rng = np.random.default_rng(2024)
    sample = np.concatenate([[0, n - 1], rng.choice(n, 150, replace=False)])
    ref = oracle_events(proc, phys, opdf, grid, 0, iteration=5, events=sample)
    assert np.array_equal(ev["bins"].cpu().numpy()[sample], ref["bins"])
    mk = ev["mask"].cpu().numpy()[sample].astype(int)
    for i in np.nonzero(mk != ref["mask"])[0]:
        assert cut_margin(proc, phys, ref["plab"][i]) < 1e-9
    same = mk == ref["mask"]
    assert_fp_parity(rel_err(w[sample][same], ref["w"][same]), 1, "w (full size, sampled)")
    assert_fp_parity(rel_err(ev["me2"].cpu().numpy()[sample][same], ref["me2"][same]), 1, "me2 (full size, sampled)")
    ctx.close()


def test_philox_counter_crosses_32_bits(pdf_grid, opdf):
    """Event numbers across 2^32 (the counter's second word) and a large
    iteration number: the random stream stays bit-exact."""
    proc = IN.GG_TT
    phys = PHYS[proc]
    grid = random_grid(IN.DIM[proc], seed=9)
    ctx = ctx_for(proc, 0, pdf_grid)
    g = torch.tensor(grid, device="cuda")
    off = (1 << 32) - 40
    sums, ev = ctx.vegas_pass(proc, phys.sqrt_s, g, 80, ev_offset=off, iteration=70000, want_events=True,
                              fields=("u", "x", "bins"))
    ref = oracle_events(proc, phys, opdf, grid, 80, iteration=70000, first=off)
    assert np.array_equal(ev["u"].cpu().numpy(), ref["u"])
    assert np.array_equal(ev["x"].cpu().numpy(), ref["x"])
    assert np.array_equal(ev["bins"].cpu().numpy(), ref["bins"])
    ctx.close()


@pytest.mark.parametrize("n_bins", [2, 64])
def test_bin_count_extremes(n_bins, pdf_grid, opdf):
    """The smallest and largest VEGAS grids: integrate e+ e- -> mu+ mu- and
    compare with the oracle's integrate at the same bin count."""
    import dataclasses
    from paper_2105_10529_gb300.api import Context
    proc = IN.EE_MUMU
    phys = dataclasses.replace(PHYS[proc], n_bins=n_bins)
    ctx = Context(phys, pdf_grid, precision=0)
    r = ctx.integrate(proc, phys.sqrt_s, 20000, 3, want_grid=True)
    ref = O.integrate(proc, phys, opdf, 20000, 3)
    assert r["sigma"] == pytest.approx(ref["sigma"], rel=1e-9)
    assert np.abs(r["grid"] - ref["grid"]).max() < 1e-9
    ctx.close()


@pytest.mark.parametrize("proc", [IN.GG_TTG, IN.GG_TTGG])
def test_stored_kinematics_match_recompute(proc, pdf_grid):
    """In mixed precision the heavy integrand keeps the kinematics of queued
    events (shared memory for g g -> t tbar g, a global per-CTA store for
    g g -> t tbar g g); the pass that recomputes them (the one with per-event
    outputs) gives the same sums up to the last bits: the two passes are
    separately compiled kernels, whose floating-point contraction of the FP64
    kinematics may differ (a wrong stored value would show as an O(1)
    difference)."""
    phys = PHYS[proc]
    grid = torch.tensor(random_grid(IN.DIM[proc], seed=41), device="cuda")
    ctx = ctx_for(proc, 1, pdf_grid)
    for sched in (0, 1, 2, 3):
        ctx.set_schedule(sched)
        n = 20011 if proc == IN.GG_TTG else 3001
        a, _ = ctx.vegas_pass(proc, phys.sqrt_s, grid, n, iteration=6)
        b, _ = ctx.vegas_pass(proc, phys.sqrt_s, grid, n, iteration=6, want_events=True, fields=("w",))
        rel = float(((a - b).abs() / b.abs().clamp_min(1e-300)).max())
        # FP64 kinematics: a few ulp; the tensor-core kernels also round FP32 apart; schedule 3
        # of g g -> t tbar g g writes its outputs from the kernel that runs without them: equal
        if sched == 3 and proc == IN.GG_TTGG:
            assert torch.equal(a, b)
            continue
        tol = 1e-14 if sched < 2 else 1e-9
        assert rel < tol, (sched, rel)
    ctx.close()


@pytest.mark.parametrize("proc", [IN.GG_TTG, IN.GG_TTGG])
def test_helicity_split_pass(proc, pdf_grid, opdf):
    """Two threads per event, each summing half of the helicities: under the
    barrier schedules the pass sums agree with one thread per event to FP32
    rounding of the two summation orders (every entry, histogram included),
    and the sum of weights with the oracle's sum over the same events."""
    phys = PHYS[proc]
    n = 1001 if proc == IN.GG_TTGG else 5003    # several batches and a ragged tail
    g = random_grid(IN.DIM[proc], seed=51)
    grid = torch.tensor(g, device="cuda")
    ctx = ctx_for(proc, 1, pdf_grid)
    scheds = (1, 2) if proc == IN.GG_TTGG else (1,)
    ref = oracle_events(proc, phys, opdf, g, n, iteration=3)
    ref_sum = float(np.sum(ref["w"])) / n
    for sched in scheds:
        ctx.set_schedule(sched)
        ctx.set_helicity_split(1)
        a, _ = ctx.vegas_pass(proc, phys.sqrt_s, grid, n, iteration=3)
        ctx.set_helicity_split(2)
        b, _ = ctx.vegas_pass(proc, phys.sqrt_s, grid, n, iteration=3)
        ctx.device_status()
        assert torch.all((a - b).abs() <= 1e-6 * a.abs() + 1e-300), sched
        assert float(b[0]) == pytest.approx(ref_sum, rel=1e-5), sched
        # the split kernel's own per-event outputs against the oracle, event by event
        c, ev = ctx.vegas_pass(proc, phys.sqrt_s, grid, n, iteration=3, want_events=True,
                               fields=("bins", "mask", "w", "me2"))
        ctx.device_status()
        assert torch.equal(b, c), sched
        check_events_against_oracle(proc, phys, opdf, g, ev, 3, 1, what=f"split 2, schedule {sched}")
    from paper_2105_10529_gb300._lib import MfError
    ctx.set_helicity_split(1)
    with pytest.raises(MfError):
        ctx.set_helicity_split(3)
    ctx.close()


def test_helicity_split_integrate(pdf_grid):
    """Iterated VEGAS of g g -> t tbar g g with the helicity split (which runs the
    tensor-core schedule 2 under the default schedule 3) agrees with no split to
    rounding; so do the per-event outputs, which the split kernel writes."""
    proc = IN.GG_TTGG
    phys = PHYS[proc]
    ctx = ctx_for(proc, 1, pdf_grid)
    r1 = ctx.integrate(proc, phys.sqrt_s, 20000, 2)
    ctx.set_helicity_split(2)
    r2 = ctx.integrate(proc, phys.sqrt_s, 20000, 2)
    ctx.device_status()
    assert r2["sigma"] == pytest.approx(r1["sigma"], rel=1e-6)
    assert r2["n_pass"] == r1["n_pass"]
    grid = torch.tensor(random_grid(IN.DIM[proc], seed=52), device="cuda")
    _, e2 = ctx.vegas_pass(proc, phys.sqrt_s, grid, 300, iteration=1, want_events=True, fields=("me2",))
    ctx.set_helicity_split(1)
    _, e1 = ctx.vegas_pass(proc, phys.sqrt_s, grid, 300, iteration=1, want_events=True, fields=("me2",))
    m1, m2 = e1["me2"].cpu().numpy(), e2["me2"].cpu().numpy()
    assert np.array_equal(m1 == 0, m2 == 0)
    nz = m1 != 0
    assert np.all(np.abs(m2[nz] - m1[nz]) <= 1e-6 * np.abs(m1[nz]))
    ctx.close()


def test_bounded_wait_expiry_is_reported(pdf_grid):
    """A device wait on an mbarrier phase that nothing completes runs out after
    its iteration limit; the host sees MF_ERR_TIMEOUT once, and the context
    keeps working."""
    proc = IN.GG_TT
    phys = PHYS[proc]
    ctx = ctx_for(proc, 1, pdf_grid)
    assert ctx.selftest_wait(2048) == 3
    ctx.device_status()                      # the flag was cleared
    g = torch.tensor(random_grid(IN.DIM[proc], seed=3), device="cuda")
    s, _ = ctx.vegas_pass(proc, phys.sqrt_s, g, 1000)
    ctx.device_status()
    assert float(s[0]) > 0.0
    ctx.close()

"""Batched channels (mf_integrate_batch): several partonic subprocesses in
one persistent launch per VEGAS iteration, each on its own grid and Philox
channel id.  Checked against the FP64 oracle channel by channel, against the
single-process path, and for independence of the CTA schedule."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from paper_2105_10529_gb300._lib import MfError

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PHYS = IN.Physics(seed=7, channel=2)
CHANNELS = [IN.GG_TT, IN.UU_TT, IN.UG_TTU, IN.GG_TTG, IN.GG_TTGG]
# uneven sizes, none a multiple of the tile
N_EV = [20011, 8003, 4001, 2503, 509]
TILE = 1000


@pytest.fixture(scope="module")
def pdf_grid():
    return IN.make_pdf_grid()


@pytest.fixture(scope="module")
def opdf(pdf_grid):
    return O.Pdf(pdf_grid)


@pytest.fixture(scope="module")
def ctx(pdf_grid):
    from paper_2105_10529_gb300.api import Context
    c = Context(PHYS, pdf_grid, precision=1)
    yield c
    c.close()


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_batch_one_iteration_matches_oracle(ctx, opdf, mode):
    """One iteration at the uniform grid: channel i is the oracle pass of that
    process with channel id PHYS.channel + i (mixed precision: 1e-5)."""
    ctx.set_batch_schedule(mode, 1, TILE, 3 * TILE, 0)
    tot, chans = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 1)
    s_sum, v_sum = 0.0, 0.0
    for i, (p, n) in enumerate(zip(CHANNELS, N_EV)):
        ph = dataclasses.replace(PHYS, channel=PHYS.channel + i)
        ref = O.vegas_pass(p, ph, opdf, O.vegas_init(IN.DIM[p], PHYS.n_bins), n)
        var = (n * ref["sum_w2"] - ref["sum_w"] ** 2) / (n - 1)
        c = chans[i]
        assert abs(c["sigma"] - ref["sum_w"]) <= 1e-5 * abs(ref["sum_w"]), (p, c["sigma"], ref["sum_w"])
        assert abs(c["error"] - np.sqrt(var)) <= 1e-5 * np.sqrt(var), (p, c["error"], np.sqrt(var))
        # events near a cut threshold may flip; none expected at these sizes
        assert abs(c["n_pass"] - ref["n_pass"]) <= 1, (p, c["n_pass"], ref["n_pass"])
        assert c["n_events"] == n and c["n_nan"] == 0
        s_sum += c["sigma"]; v_sum += c["error"] ** 2
    assert tot["sigma"] == pytest.approx(s_sum, rel=1e-15)
    assert tot["error"] == pytest.approx(np.sqrt(v_sum), rel=1e-15)
    assert tot["n_events"] == sum(N_EV)


# (mode, barrier schedule, helicity split): the persistent kernel with and without the barrier and
# the split, the split mode (heavy channels persistent, the others as their own kernels), and the
# per-channel kernels with the warp-per-event schedules (diagrams, helicity-recycled recursion)
@pytest.mark.parametrize("mode,sched,hsplit", [(0, 0, 1), (0, 1, 2), (1, 1, 1), (2, 3, 1), (2, 4, 1), (3, 4, 1)])
def test_batch_pass_events_match_oracle(ctx, opdf, mode, sched, hsplit):
    """One batch pass at non-uniform caller grids with per-event outputs,
    written by the batch's own kernels (the persistent kernel in modes 0 and
    1): every channel's events against the oracle's, bins bit-exact and w,
    |M|^2 within the mixed-precision bound, and the channel's pass sums equal
    to the sums of its per-event weights and to the pass without outputs."""
    from tests.gpu_common import check_events_against_oracle, random_grid
    n_ev = [3001, 2003, 1201, 601, 151]
    nb = PHYS.n_bins
    grids = np.zeros((len(CHANNELS), 18, nb + 1))
    for i, p in enumerate(CHANNELS):
        grids[i, :IN.DIM[p]] = random_grid(IN.DIM[p], nb, seed=90 + i)
    gt = torch.tensor(grids, device="cuda")
    ctx.set_batch_schedule(mode, sched, 256, 512, 0, hsplit)
    plain, _ = ctx.batch_pass(CHANNELS, n_ev, PHYS.sqrt_s, gt, iteration=6)
    sums, evs = ctx.batch_pass(CHANNELS, n_ev, PHYS.sqrt_s, gt, iteration=6, want_events=True,
                               fields=("bins", "mask", "w", "me2"))
    ctx.device_status()
    assert torch.equal(plain, sums)
    for i, (p, n) in enumerate(zip(CHANNELS, n_ev)):
        ph = dataclasses.replace(PHYS, channel=PHYS.channel + i)
        w = evs[i]["w"].cpu().numpy()
        s0 = float(sums[i, 0])
        assert abs(s0 - w.sum() / n) <= 1e-12 * abs(w.sum() / n) + 1e-300, p
        check_events_against_oracle(p, ph, opdf, grids[i, :IN.DIM[p]], evs[i], 6, 1,
                                    what=f"batch mode {mode} sched {sched} split {hsplit} process {p}")


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_batch_iterations_match_single_process(ctx, pdf_grid, mode):
    """Three iterations with refinement: each channel equals mf_integrate of
    that process alone (same channel id); only the grouping of the sums
    differs (tiles against CTAs)."""
    from paper_2105_10529_gb300.api import Context
    ctx.set_batch_schedule(mode, 1, TILE, 3 * TILE, 0)
    tot, chans = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 3, want_grids=True)
    for i, (p, n) in enumerate(zip(CHANNELS, N_EV)):
        single = Context(dataclasses.replace(PHYS, channel=PHYS.channel + i), pdf_grid, precision=1)
        single.set_schedule(1)      # the batch sums colour flows with FP32 FMAs
        r = single.integrate(p, PHYS.sqrt_s, n, 3, want_grid=True)
        single.close()
        assert chans[i]["sigma"] == pytest.approx(r["sigma"], rel=1e-9), p
        assert chans[i]["error"] == pytest.approx(r["error"], rel=1e-7), p
        assert chans[i]["n_pass"] == r["n_pass"], p
        assert np.abs(chans[i]["grid"] - r["grid"]).max() < 1e-9, p


def test_batch_light_channels_match_oracle_integrate(ctx, opdf):
    """Iterated VEGAS of the light channels against the oracle's integrate."""
    procs, ns = [IN.GG_TT, IN.UU_TT], [30001, 12001]
    ctx.set_batch_schedule(0, 0, 2048, 2048, 0)
    tot, chans = ctx.integrate_batch(procs, ns, PHYS.sqrt_s, 3)
    for i, (p, n) in enumerate(zip(procs, ns)):
        ref = O.integrate(p, dataclasses.replace(PHYS, channel=PHYS.channel + i), opdf, n, 3)
        assert chans[i]["sigma"] == pytest.approx(ref["sigma"], rel=1e-5), p
        assert chans[i]["error"] == pytest.approx(ref["error"], rel=1e-4), p


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_batch_schedule_independent(ctx, mode):
    """At fixed mode and tile sizes the result is bit-identical for every
    barrier schedule and CTA count, and on repeated (graph-replayed) calls."""
    ref = None
    for sched, bps in [(1, 0), (0, 0), (1, 1), (0, 2), (1, 0)]:
        ctx.set_batch_schedule(mode, sched, TILE, 3 * TILE, bps)
        tot, chans = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 2, want_grids=True)
        key = [(c["sigma"], c["error"], c["n_pass"]) for c in chans]
        grids = [c["grid"] for c in chans]
        if ref is None:
            ref = (key, grids)
        else:
            assert key == ref[0], (sched, bps)
            for a, b in zip(grids, ref[1]):
                assert np.array_equal(a, b)


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_helicity_split(ctx, mode):
    """The helicity split of the g g -> t tbar g(g) channels changes the
    summation order only: every channel within 1e-6 of no split, same counts."""
    ctx.set_batch_schedule(mode, 1, TILE, 3 * TILE, 0, 1)
    t1, c1 = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 2)
    ctx.set_batch_schedule(mode, 1, TILE, 3 * TILE, 0, 2)
    t2, c2 = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 2)
    for a, b in zip(c1, c2):
        assert b["sigma"] == pytest.approx(a["sigma"], rel=1e-6)
        assert b["n_pass"] == a["n_pass"]
    assert t2["sigma"] == pytest.approx(t1["sigma"], rel=1e-6)
    ctx.set_batch_schedule(mode, 1, TILE, 3 * TILE, 0)


@pytest.mark.parametrize("sched", [2, 3, 4])
def test_batch_per_channel_kernels_with_tensor_cores(sched, ctx, pdf_grid):
    """Mode 2 with the tensor-core colour sum (integrand schedule 2), with the
    warp-per-event schedule (3) and with the helicity-recycled recursion (4):
    each channel equals a single-process
    mf_integrate on the same integrand schedule (the same kernels and launch
    configuration), and the result is stable under graph replay."""
    from paper_2105_10529_gb300.api import Context
    ctx.set_batch_schedule(2, sched, TILE, 3 * TILE, 0)
    tot, chans = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 2)
    tot2, chans2 = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 2)
    assert [c["sigma"] for c in chans] == [c["sigma"] for c in chans2]
    for i, (p, n) in enumerate(zip(CHANNELS, N_EV)):
        single = Context(dataclasses.replace(PHYS, channel=PHYS.channel + i), pdf_grid, precision=1)
        single.set_schedule(sched)
        r = single.integrate(p, PHYS.sqrt_s, n, 2)
        single.close()
        assert chans[i]["sigma"] == pytest.approx(r["sigma"], rel=1e-9), p
        assert chans[i]["n_pass"] == r["n_pass"], p
    ctx.set_batch_schedule(1, 1, TILE, 3 * TILE, 0)


def test_batch_graph_cache_invalidation(ctx):
    """A different channel list in between re-captures; the original list
    then gives the same numbers again."""
    ctx.set_batch_schedule(1, 1, TILE, 3 * TILE, 0)
    a, ca = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 2)
    b, cb = ctx.integrate_batch([IN.GG_TT], [5003], PHYS.sqrt_s, 2)
    assert cb[0]["n_events"] == 2 * 5003
    a2, ca2 = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 2)
    assert [c["sigma"] for c in ca] == [c["sigma"] for c in ca2]
    # the same process twice: different channel ids, different streams
    d, cd = ctx.integrate_batch([IN.GG_TT, IN.GG_TT], [5003, 5003], PHYS.sqrt_s, 1)
    assert cd[0]["sigma"] != cd[1]["sigma"]
    assert cd[0]["sigma"] == pytest.approx(cd[1]["sigma"], rel=0.1)


def test_batch_autotune(ctx):
    choice = ctx.autotune_batch(CHANNELS, [40000, 10000, 10000, 8000, 4000], PHYS.sqrt_s)
    # the candidates: modes 0/1 with heavy tiles 1024/2048/4096 and light tiles 2048/4096; mode 2
    # with heavy tiles 512/4096 and light tiles 256/2048/4096; mode 3 (schedule 4) with heavy tiles
    # 512/4096 and light tiles 256/2048
    assert choice[0] in (0, 1, 2, 3) and choice[1] in (0, 1, 2, 3, 4)
    assert choice[2] in ((512, 4096) if choice[0] >= 2 else (1024, 2048, 4096))
    assert choice[1] < 2 or choice[0] >= 2
    assert choice[0] != 3 or choice[1] == 4
    assert choice[3] in ({2: (256, 2048, 4096), 3: (256, 2048)}.get(choice[0], (2048, 4096)))
    assert choice[4] == 0 and choice[5] in (1, 2)
    assert choice[5] == 1 or choice[1] == 1
    tot, chans = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 1)
    ctx.set_batch_schedule(*choice)
    tot2, chans2 = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 1)
    assert [c["sigma"] for c in chans] == [c["sigma"] for c in chans2]


def test_batch_bad_arguments(ctx, pdf_grid):
    from paper_2105_10529_gb300.api import Context
    for procs, ns in [([], []), ([IN.GG_TT] * 9, [100] * 9), ([IN.EE_MUMU], [100]), ([IN.GG_TT], [1]),
                      ([17], [100])]:
        with pytest.raises(MfError) as e:
            ctx.integrate_batch(procs, ns, PHYS.sqrt_s, 1)
        assert e.value.code == 1, procs
    with pytest.raises(MfError) as e:
        ctx.integrate_batch([IN.GG_TT], [100], PHYS.sqrt_s, 0)
    assert e.value.code == 1
    for bad in [(1, 2, 1024, 4096, 0), (1, 1, 16, 4096, 0), (1, 1, 1024, 16, 0),
                (1, 1, 1024, 4096, -1), (1, 1, 1024, 4096, 0, 3), (1, 0, 1024, 4096, 0, 2), (4, 1, 1024, 4096, 0),
                (3, 1, 1024, 4096, 0, 2),
                (0, 2, 1024, 4096, 0), (2, 1, 1024, 4096, 0, 2), (1, 3, 1024, 4096, 0), (2, 5, 1024, 4096, 0)]:
        with pytest.raises(MfError):
            ctx.set_batch_schedule(*bad)
    f64 = Context(PHYS, pdf_grid, precision=0)
    with pytest.raises(MfError) as e:
        f64.integrate_batch([IN.GG_TT], [100], PHYS.sqrt_s, 1)
    assert e.value.code == 5
    f64.close()


def test_batch_grad_matches_single_process(ctx, pdf_grid):
    """d sigma_total/d m_t: per channel equal to mf_vegas_pass_grad of that
    process at the batch's final grid (same kernel, same channel id), and the
    total is the sum over channels."""
    from paper_2105_10529_gb300.api import Context
    ctx.set_batch_schedule(1, 1, TILE, 3 * TILE, 0)
    tot, chans = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 2, want_grids=True)
    it = 7
    g = ctx.batch_grad(CHANNELS, N_EV, PHYS.sqrt_s, it)
    for i, (p, n) in enumerate(zip(CHANNELS, N_EV)):
        single = Context(dataclasses.replace(PHYS, channel=PHYS.channel + i), pdf_grid, precision=1)
        o = single.vegas_pass_grad(p, PHYS.sqrt_s, torch.tensor(chans[i]["grid"], device="cuda"), n,
                                   iteration=it).cpu().numpy()
        single.close()
        assert g[i, 0] == o[0] and g[i, 1] == o[1] and g[i, 3] == o[3], p
        var = (n * o[2] - o[1] ** 2) / (n - 1)
        assert g[i, 2] == pytest.approx(np.sqrt(var), rel=1e-12)
        # the top mass derivative of a top-pair rate is negative
        assert g[i, 1] < 0.0, p
    assert g[-1, 0] == pytest.approx(g[:-1, 0].sum(), rel=1e-14)
    assert g[-1, 1] == pytest.approx(g[:-1, 1].sum(), rel=1e-14)
    assert g[-1, 2] == pytest.approx(np.sqrt((g[:-1, 2] ** 2).sum()), rel=1e-14)
    with pytest.raises(MfError):
        ctx.batch_grad([IN.GG_TT], [100], PHYS.sqrt_s, it)
    # want_grads in the batch call: the same passes on Philox iteration n_iter
    tot2, chans2 = ctx.integrate_batch(CHANNELS, N_EV, PHYS.sqrt_s, 2, want_grads=True)
    g2 = ctx.batch_grad(CHANNELS, N_EV, PHYS.sqrt_s, 2)
    for i in range(len(CHANNELS)):
        assert chans2[i]["dsigma_dmt"] == g2[i, 1] and chans2[i]["dsigma_dalphas"] == g2[i, 3]
        assert chans2[i]["dsigma_dmt_error"] == g2[i, 2]
    assert tot2["dsigma_dmt"] == g2[-1, 1] and tot2["dsigma_dmt_error"] == g2[-1, 2]

"""Throughput benchmark of the leading-order integrand (one JSON line on stdout).

A step is one VEGAS iteration of the g g -> t tbar g g integrand at 13 TeV
(4e6 events: Philox -> VEGAS map -> parton map -> RAMBO -> cuts -> PDF ->
|M|^2 with 123 diagrams, 64 helicities, 24 colour flows -> weights and
histograms -> grid refinement), mixed FP32/FP64 precision, on synthetic
inputs.  The FP64 GPU path, the per-event error of the mixed path and the
FP64 CPU oracle are measured in the same run.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank processes its own block of events
(weak scaling); the per-iteration pass sums are all-reduced before every
rank refines the same grid.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK = 6800.0
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
FP64_PEAK_NOMINAL_TFLOPS = 1.25
# DRAM bytes (read + write) per event of the mixed g g -> t tbar g g integrand, from the
# dram__bytes counters of 1e6-event ncu captures: schedule 3 (diagram helicity body, one lane
# per helicity; profiles/integrand_gg_ttgg_mixed_1m_ncu.txt: evicted local-memory lines, which
# grow with the number of events) and schedule 4, the default (helicity-recycled recursion;
# profiles/integrand_gg_ttgg_recycled_1m_ncu.txt: no spills; the per-CTA records and sums, and
# the out-of-line double-float kinematics' results passed through the stack, partly evicted
# from L2)
DRAM_BYTES_PER_EVENT_P3 = 4235.4
DRAM_BYTES_PER_EVENT_P4 = 109.9
DEFAULT_SCHED = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--events", type=int, default=4_000_000)
    ap.add_argument("--fp64-events", type=int, default=200_000)
    ap.add_argument("--oracle-err-events", type=int, default=100_000,
                    help="events of the mixed pass recomputed by the FP64 CPU oracle for the stated per-event error")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched p p -> t tbar + jets leg")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the legs that run the other single-process workloads at full size and time "
                         "the derivative and evaluate calls")
    ap.add_argument("--batch-iters", type=int, default=10)
    ap.add_argument("--ttggg-events", type=int, default=400_000,
                    help="events of the timed mixed-precision g g -> t tbar g g g pass")
    ap.add_argument("--sched", type=int, default=None,
                    help="integrand schedule (0 free warps, 1 CTA barrier per helicity, 2 = 1 + colour sum on the "
                         "tensor cores, 3 = 2 with one warp per event and one lane per helicity, 4 = one warp per "
                         "event with the helicity-recycled recursion (g g -> t tbar g g; else as 3); default 4)")
    ap.add_argument("--hsplit", type=int, default=None,
                    help="threads per event of the heavy integrand (1 or 2; default 1)")
    ap.add_argument("--only-timed", action="store_true",
                    help="run only the warm-up and timed mixed-precision steps (for profiler captures)")
    ap.add_argument("--only-grad", action="store_true",
                    help="run only the derivative calls of --process in mixed precision (for profiler captures): "
                         "d|M|^2/dp of --events points from one pass, then the m_t pass of --events events, each "
                         "once untimed and once timed")
    ap.add_argument("--process", default="gg_ttgg",
                    choices=["gg_tt", "uu_tt", "gg_ttg", "ug_ttu", "gg_ttgg", "gg_ttggg"],
                    help="process of the timed steps with --only-timed (the benchmark line is gg_ttgg)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": HBM_FALLBACK, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, index: int):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")
        try:
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if sm:
            sm.sort()
            out = {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def flops_per_event_me(process: int, sched: int = DEFAULT_SCHED) -> float:
    """Algorithmic FLOPs of the matrix element per event passing the cuts, of the method the
    schedule runs: the helicity-recycled recursion (g g -> t tbar g g, schedule 4) or the
    Feynman-diagram helicity body (parity-halved helicity sum)."""
    from fractions import Fraction
    from paper_2105_10529_gb300.gen import qcd_diagrams as Q, rc_tables as RT
    if process == 5 and sched == 4:
        return float(RT.flops_per_event(RT.build())["total"])
    k = {1: 2, 3: 3, 5: 4}[process]
    _, st = Q.generate_gluon_process(k, "x", Fraction(1))
    return float(st["flops_me"])


def run_batch(ctx, phys, IN, n_iter):
    """mf_integrate_batch over the channels of p p -> t tbar + jets: autotuned
    schedule, one warm-up call (graph capture), one timed call of n_iter
    iterations; the same channels one at a time through mf_integrate for
    comparison; d sigma_total / d m_t at the final grids."""
    procs = [p for p, _ in IN.BATCH_CHANNELS]
    ns = [int(n) for _, n in IN.BATCH_CHANNELS]
    names = {IN.GG_TT: "gg_tt", IN.UU_TT: "uu_tt", IN.GG_TTG: "gg_ttg", IN.UG_TTU: "ug_ttu", IN.GG_TTGG: "gg_ttgg"}
    choice = ctx.autotune_batch(procs, ns, phys.sqrt_s)

    def timed(sch):
        ctx.set_batch_schedule(*sch)
        ctx.integrate_batch(procs, ns, phys.sqrt_s, n_iter)          # graph capture
        t0 = time.perf_counter()
        r = ctx.integrate_batch(procs, ns, phys.sqrt_s, n_iter)
        return time.perf_counter() - t0, r

    # the chosen schedule, and one representative schedule per mode
    t_batch, (tot, chans) = timed(choice)
    per_mode = {0: timed((0, 1, 4096, 4096, 0, 1)), 1: timed((1, 1, 4096, 4096, 0, 1)),
                2: timed((2, 3, 4096, 4096, 0, 1)), 3: timed((3, 4, 4096, 2048, 0, 1))}
    ctx.set_batch_schedule(*choice)
    ctx.integrate_batch(procs, ns, phys.sqrt_s, n_iter)               # grids of the chosen schedule
    g = ctx.batch_grad(procs, ns, phys.sqrt_s, 1000)
    seq, t_ch = [], []
    for p, n in zip(procs, ns):
        t0 = time.perf_counter()
        seq.append(ctx.integrate(p, phys.sqrt_s, n, n_iter))
        t_ch.append(time.perf_counter() - t0)
    t_seq = sum(t_ch)
    ev = sum(ns) * n_iter
    return {"workload": "p p -> t tbar + jets: " + ", ".join(f"{names[p]} {n:.0e}" for p, n in zip(procs, ns))
                        + f" events per iteration, {n_iter} iterations, mixed precision",
            "events_per_s": ev / t_batch, "s_per_call": t_batch,
            "sequential_events_per_s": ev / t_seq, "speedup_vs_sequential": t_seq / t_batch,
            "sequential_s_by_channel": {names[p]: t for p, t in zip(procs, t_ch)},
            "schedule": {"mode": ["one launch", "split", "per-channel kernels",
                                  "per-channel kernels in turn"][choice[0]],
                         "integrand_schedule": choice[1],
                         "tile_heavy": choice[2], "tile_light": choice[3], "ctas_per_sm": choice[4],
                         "helicity_split": choice[5]},
            "events_per_s_by_mode": {"one launch (0, 1, 4096, 4096)": ev / per_mode[0][0],
                                     "split (1, 1, 4096, 4096)": ev / per_mode[1][0],
                                     "per-channel kernels (2, 3, -, 4096)": ev / per_mode[2][0],
                                     "per-channel kernels in turn (3, 4, -, 2048)": ev / per_mode[3][0]},
            "sigma_pb": tot["sigma"], "error_pb": tot["error"],
            "channels": {names[p]: {"sigma_pb": c["sigma"], "error_pb": c["error"], "chi2dof": c["chi2dof"],
                                    "sequential_sigma_pb": q["sigma"]} for p, c, q in zip(procs, chans, seq)},
            "dsigma_dmt_pb_per_gev": float(g[-1, 1]), "dsigma_dmt_error": float(g[-1, 2]),
            "dsigma_dalphas_pb": float(g[-1, 3]),
            "timing": "host wall clock around the synchronous C-ABI call (graph launch, reductions, host results)",
            "small_channels": run_small_batch(ctx, phys, IN)}


def run_small_batch(ctx, phys, IN, n_iter=5, reps=5):
    """Many small, uneven channels (eight channels of 5e3 .. 6e4 events, five iterations):
    where launch gaps and per-kernel tails dominate, one graph-replayed batch call against
    the same channels one mf_integrate call after another (each itself graph-replayed);
    best of reps calls each, after warm-up calls, autotuned batch schedule."""
    procs = [IN.GG_TT, IN.UU_TT, IN.GG_TTG, IN.UG_TTU, IN.GG_TTGG, IN.GG_TT, IN.UG_TTU, IN.GG_TTG]
    ns = [60000, 20000, 30000, 10000, 5000, 40000, 15000, 8000]
    choice = ctx.autotune_batch(procs, ns, phys.sqrt_s)
    ctx.set_batch_schedule(*choice)
    ctx.integrate_batch(procs, ns, phys.sqrt_s, n_iter)
    t_b = []
    for _ in range(reps):
        t0 = time.perf_counter()
        ctx.integrate_batch(procs, ns, phys.sqrt_s, n_iter)
        t_b.append(time.perf_counter() - t0)
    for p, n in zip(procs, ns):
        ctx.integrate(p, phys.sqrt_s, n, n_iter)
    t_s = []
    for _ in range(reps):
        t0 = time.perf_counter()
        for p, n in zip(procs, ns):
            ctx.integrate(p, phys.sqrt_s, n, n_iter)
        t_s.append(time.perf_counter() - t0)
    ev = sum(ns) * n_iter
    return {"channels": len(procs), "events_per_iteration": ns, "iterations": n_iter,
            "batch_events_per_s": ev / min(t_b), "sequential_events_per_s": ev / min(t_s),
            "speedup_vs_sequential": min(t_s) / min(t_b), "schedule": list(choice)}


def run_configs(pdf, IN, MF_FP64, MF_MIXED, stream):
    """The other single-process workloads at their full sizes through
    mf_integrate (host wall clock around the synchronous call, one warm-up
    call first): e+e- -> mu+mu- in FP64 (1e5 x 5); g g -> t tbar and
    g g -> t tbar g (1e7 x 10) in mixed precision and in FP64, the latter with
    d sigma/d m_t from the extra derivative pass; and the per-event relative
    error of the mixed weights against the FP64 GPU weights on 1e5 events at
    the uniform grid."""
    import numpy as np
    import torch
    from paper_2105_10529_gb300.api import Context, process_info
    out = {}
    names = {IN.EE_MUMU: "ee_mumu", IN.GG_TT: "gg_tt", IN.GG_TTG: "gg_ttg"}
    for key, wl in IN.workloads().items():
        p = wl.process
        if p not in names:
            continue
        grads = p == IN.GG_TTG
        precs = [MF_FP64] if p == IN.EE_MUMU else [MF_MIXED, MF_FP64]
        entry = {"workload": wl.name, "events_per_iteration": wl.n_events, "iterations": wl.n_iter}
        ws = {}
        for prec in precs:
            ctx = Context(wl.physics, pdf, precision=prec, stream=stream)
            ctx.integrate(p, wl.physics.sqrt_s, min(wl.n_events, 100_000), 1)          # warm-up
            t0 = time.perf_counter()
            r = ctx.integrate(p, wl.physics.sqrt_s, wl.n_events, wl.n_iter, want_grads=grads)
            dt = time.perf_counter() - t0
            tag = "fp64" if prec == MF_FP64 else "mixed"
            e = {"events_per_s": wl.n_events * wl.n_iter / dt, "s_per_call": dt, "sigma_pb": r["sigma"],
                 "error_pb": r["error"], "chi2dof": r["chi2dof"], "pass_fraction": r["n_pass"] / max(r["n_events"], 1)}
            if grads:
                e.update(dsigma_dmt_pb_per_gev=r["dsigma_dmt"], dsigma_dmt_error=r["dsigma_dmt_error"],
                         dsigma_dalphas_pb=r["dsigma_dalphas"],
                         timing_note="includes one derivative pass of the same size at the final grid")
            entry[tag] = e
            if len(precs) > 1:
                _, dim = process_info(p)
                grid = torch.linspace(0, 1, wl.physics.n_bins + 1, dtype=torch.float64,
                                      device="cuda").repeat(dim, 1).contiguous()
                _, ev = ctx.vegas_pass(p, wl.physics.sqrt_s, grid, 100_000, iteration=10**6, want_events=True,
                                       fields=("w",))
                torch.cuda.synchronize()
                ws[tag] = ev["w"].cpu().numpy()
            ctx.close()
        if "mixed" in entry and "fp64" in entry:
            ok = ws["fp64"] != 0
            rel = np.abs(ws["mixed"][ok] - ws["fp64"][ok]) / np.abs(ws["fp64"][ok])
            entry["mixed_speedup"] = entry["mixed"]["events_per_s"] / entry["fp64"]["events_per_s"]
            entry["stated_err"] = {"per_event_rel_max": float(rel.max()),
                                   "per_event_rel_p999": float(np.quantile(rel, 0.999)),
                                   "per_event_rel_median": float(np.median(rel)), "events": int(ok.sum()),
                                   "sigma_rel_mixed_vs_fp64": abs(entry["mixed"]["sigma_pb"] - entry["fp64"]["sigma_pb"])
                                   / abs(entry["fp64"]["sigma_pb"])}
        out[names[p]] = entry
    return out


def run_derivatives(ctx, phys, IN, grid, stream):
    """Rates of the derivative and evaluate calls (mixed precision, CUDA events
    on the stream, one warm-up call each): the m_t-derivative pass of the
    estimator (mf_vegas_pass_grad) for g g -> t tbar g and g g -> t tbar g g at
    their full pass sizes and the adapted g g -> t tbar g g grid, and
    mf_evaluate of g g -> t tbar g g momenta with and without d|M|^2/dp."""
    import torch
    from paper_2105_10529_gb300.api import process_info

    def timed(fn):
        fn()                                       # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        res = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, res

    out = {}
    dev = grid.device
    for proc, n, name in ((IN.GG_TTG, 10_000_000, "gg_ttg"), (IN.GG_TTGG, 4_000_000, "gg_ttgg")):
        _, dim = process_info(proc)
        g = grid if proc == IN.GG_TTGG else torch.linspace(0, 1, phys.n_bins + 1, dtype=torch.float64,
                                                           device=dev).repeat(dim, 1).contiguous()
        t, r = timed(lambda: ctx.vegas_pass_grad(proc, phys.sqrt_s, g, n, iteration=77))
        tv, _ = timed(lambda: ctx.vegas_pass(proc, phys.sqrt_s, g, n, iteration=77))
        r = r.cpu().tolist()
        out[f"dsigma_dmt_pass_{name}"] = {
            "events": n, "events_per_s": n / t, "s": t, "over_value_pass": t / tv, "sigma_hat_pb": r[0],
            "dsigma_dmt_pb_per_gev": r[1], "dsigma_dalphas_pb": r[3],
            "method": ("forward mode through the helicity-recycled recursion (dual numbers), kinematics with the "
                       "m_t tangent" if proc == IN.GG_TTGG else "forward tangents through the generated diagrams")}
    n_ev = 100_000
    _, ev = ctx.vegas_pass(IN.GG_TTGG, phys.sqrt_s, grid, n_ev, ev_offset=5 * 10**8, iteration=78,
                           want_events=True, fields=("momenta",))
    mom = ev["momenta"]
    t, _ = timed(lambda: ctx.evaluate(IN.GG_TTGG, mom))
    out["evaluate_gg_ttgg"] = {"points": n_ev, "points_per_s": n_ev / t, "s": t}
    n_g = 100_000
    mg = mom[:n_g].contiguous()
    t, _ = timed(lambda: ctx.evaluate_grad(IN.GG_TTGG, mg))
    tv, _ = timed(lambda: ctx.evaluate(IN.GG_TTGG, mg))
    out["evaluate_with_dme2_dp_gg_ttgg"] = {"points": n_g, "points_per_s": n_g / t, "s": t, "over_value": t / tv,
                                            "note": "reverse sweep of the helicity-recycled recursion, tangents "
                                                    "through the invariants; over_value against the diagram "
                                                    "evaluate kernel"}
    return out


def run_helicity(pdf, IN, MF_FP64, MF_MIXED, stream):
    """Helicity measurement (mf_helicity_profile, FP64) on events that pass the
    cuts at the uniform grid, per top process: configurations in all, exactly
    zero ones (skipped by the integrand), the mean share of |M|^2 carried by the
    largest configuration and the mean number of configurations that carry
    99%; and the light-quark channels' pass time (mixed, 4e6 events, CUDA
    events) with the filtered helicity loops."""
    import numpy as np
    import torch
    from paper_2105_10529_gb300.api import Context, process_info
    out = {}
    names = {IN.GG_TT: "gg_tt", IN.UU_TT: "uu_tt", IN.GG_TTG: "gg_ttg", IN.UG_TTU: "ug_ttu", IN.GG_TTGG: "gg_ttgg"}
    for p, name in names.items():
        phys = IN.Physics(seed=11)
        _, dim = process_info(p)
        grid = torch.linspace(0, 1, phys.n_bins + 1, dtype=torch.float64, device="cuda").repeat(dim, 1).contiguous()
        ctx = Context(phys, pdf, precision=MF_FP64, stream=stream)
        _, ev = ctx.vegas_pass(p, phys.sqrt_s, grid, 4000, iteration=5, want_events=True, fields=("mask", "momenta"))
        mom = ev["momenta"][ev["mask"].bool()][:2000].contiguous()
        prof = ctx.helicity_profile(p, mom).cpu().numpy()
        ctx.close()
        tot = prof.sum(1, keepdims=True)
        share = prof / tot
        srt = -np.sort(-share, axis=1)
        n99 = (np.cumsum(srt, axis=1) < 0.99).sum(1) + 1
        entry = {"configurations": int(prof.shape[1]), "exactly_zero": int(np.all(prof == 0.0, axis=0).sum()),
                 "mean_largest_share": float(srt[:, 0].mean()), "mean_configs_for_99pct": float(n99.mean()),
                 "mean_smallest_nonzero_share": float(np.where(share > 0, share, np.inf).min(1).mean()),
                 "events": int(prof.shape[0])}
        if p in (IN.UU_TT, IN.UG_TTU):
            ctx = Context(phys, pdf, precision=MF_MIXED, stream=stream)
            ctx.vegas_pass(p, phys.sqrt_s, grid, 400_000, iteration=0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.vegas_pass(p, phys.sqrt_s, grid, 4_000_000, iteration=1)
            e1.record(stream)
            torch.cuda.synchronize()
            entry["mixed_pass_ms_4e6_filtered"] = e0.elapsed_time(e1)
            ctx.close()
        out[name] = entry
    return out


def run_ttggg(pdf, IN, MF_FP64, MF_MIXED, stream, n_mixed, fma32):
    """g g -> t tbar g g g (the multi-leg extension: 5 gluons, 120 colour orderings,
    warp-level Berends-Giele recursion): one mixed-precision pass of n_mixed events
    and one FP64 pass, CUDA events on the stream after a warm-up pass, at the grid
    after two refined iterations; the algorithmic FLOPs of the recursion per event
    that passes the cuts (64 helicity configurations); the per-event error of the
    mixed weights against the FP64 CPU oracle on a sample; sigma from 2 iterations."""
    import numpy as np
    import torch
    from paper_2105_10529_gb300.api import Context, process_info
    from paper_2105_10529_gb300.gen import bg_tables
    p = IN.GG_TTGGG
    phys = IN.workloads()["gg_ttggg"].physics
    _, dim = process_info(p)
    hel = bg_tables.helicity_flops(5)
    fl_event = 64 * hel["total"]
    out = {"workload": "g g -> t tbar g g g LO, 13 TeV, pT(g)>30, |eta(g)|<2.5, dR(g,g)>0.4 for every pair",
           "flops_per_passing_event": fl_event, "flops_basis": "bg_tables.helicity_flops(5) x 64 helicities",
           "flops_split_per_helicity": {k: v for k, v in hel.items() if k not in ("counts",)}}
    ctx = Context(phys, pdf, precision=MF_MIXED, stream=stream)
    r = ctx.integrate(p, phys.sqrt_s, 100_000, 2, want_grid=True)
    grid = torch.tensor(r["grid"], device="cuda")
    _, ev = ctx.vegas_pass(p, phys.sqrt_s, grid, 50_000, iteration=50, want_events=True, fields=("mask", "w"))
    pass_frac = float(ev["mask"].float().mean().item())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.vegas_pass(p, phys.sqrt_s, grid, 100_000, iteration=51)
    torch.cuda.synchronize()
    e0.record(stream)
    s32, _ = ctx.vegas_pass(p, phys.sqrt_s, grid, n_mixed, iteration=52)
    e1.record(stream)
    torch.cuda.synchronize()
    t32 = e0.elapsed_time(e1) / 1e3
    ach = fl_event * n_mixed * pass_frac / t32 / 1e12
    out["mixed"] = {"events": n_mixed, "events_per_s": n_mixed / t32, "kernel_ms": t32 * 1e3, "pass_fraction": pass_frac,
                    "achieved_tflops": ach, "frac_of_fp32_peak": ach / (SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ / 1e6),
                    "frac_of_measured_fma_peak": ach / fma32, "sigma_2_iterations_pb": r["sigma"],
                    "error_pb": r["error"]}
    # helicity sampling: pass time and per-event weight variance against the full sum on the
    # same events; the time to a given error scales as time x variance
    _, evf = ctx.vegas_pass(p, phys.sqrt_s, grid, 50_000, iteration=56, want_events=True, fields=("w",))
    var_full = float(evf["w"].var().item())
    samp = {}
    for ns in (8, 1):
        ctx.set_helicity_sampling(ns, 1)
        _, evs_ = ctx.vegas_pass(p, phys.sqrt_s, grid, 50_000, iteration=56, want_events=True, fields=("w",))
        var_s = float(evs_["w"].var().item())
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.vegas_pass(p, phys.sqrt_s, grid, n_mixed, iteration=52)
        e1.record(stream)
        torch.cuda.synchronize()
        ts = e0.elapsed_time(e1) / 1e3
        samp[str(ns)] = {"events_per_s": n_mixed / ts, "speedup": t32 / ts, "weight_variance_ratio": var_s / var_full,
                         "time_to_equal_error_gain": (t32 / ts) / (var_s / var_full)}
    ctx.set_helicity_sampling(0)
    out["mixed"]["helicity_sampling"] = {"configurations_of_64": samp, "variance_sample_events": 50_000}
    # derivatives: the m_t pass (forward mode through the recursion) and d|M|^2/dp (reverse sweep)
    n_d = max(4000, n_mixed // 10)
    ctx.vegas_pass_grad(p, phys.sqrt_s, grid, 2000, iteration=57)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.vegas_pass_grad(p, phys.sqrt_s, grid, n_d, iteration=58)
    e1.record(stream)
    torch.cuda.synchronize()
    td = e0.elapsed_time(e1) / 1e3
    e0.record(stream)
    ctx.vegas_pass(p, phys.sqrt_s, grid, n_d, iteration=58)
    e1.record(stream)
    torch.cuda.synchronize()
    tvd = e0.elapsed_time(e1) / 1e3
    _, evm = ctx.vegas_pass(p, phys.sqrt_s, grid, 4 * 4000, iteration=59, want_events=True, fields=("mask", "momenta"))
    mom = evm["momenta"][evm["mask"].bool()][:4000].contiguous()
    ctx.evaluate_grad(p, mom)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.evaluate_grad(p, mom)
    e1.record(stream)
    torch.cuda.synchronize()
    tg = e0.elapsed_time(e1) / 1e3
    e0.record(stream)
    ctx.evaluate(p, mom)
    e1.record(stream)
    torch.cuda.synchronize()
    te = e0.elapsed_time(e1) / 1e3
    out["derivatives"] = {"dsigma_dmt_pass": {"events": n_d, "events_per_s": n_d / td, "over_value_pass": td / tvd,
                                              "method": "forward mode through the recursion (dual numbers)"},
                          "evaluate_with_dme2_dp": {"points": int(mom.shape[0]), "points_per_s": mom.shape[0] / tg,
                                                    "over_value": tg / te, "method": "reverse sweep per helicity"}}
    ctx.close()
    n64 = max(2000, n_mixed // 50)
    ctx64 = Context(phys, pdf, precision=MF_FP64, stream=stream)
    ctx64.vegas_pass(p, phys.sqrt_s, grid, 2000, iteration=53)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx64.vegas_pass(p, phys.sqrt_s, grid, n64, iteration=54)
    e1.record(stream)
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) / 1e3
    out["fp64"] = {"events": n64, "events_per_s": n64 / t64, "mixed_speedup": (n_mixed / t32) / (n64 / t64)}
    ctx64.close()
    # per-event error of the mixed path against the FP64 CPU oracle
    try:
        import oracle as O
        n_or = 400
        ctx = Context(phys, pdf, precision=MF_MIXED, stream=stream)
        _, evm = ctx.vegas_pass(p, phys.sqrt_s, grid, n_or, iteration=55, want_events=True, fields=("w",))
        torch.cuda.synchronize()
        ctx.close()
        t0 = time.perf_counter()
        evs = O.events(p, phys, O.Pdf(pdf), grid.cpu().numpy(), range(n_or), 55, n_threads=os.cpu_count() or 1)
        t_or = time.perf_counter() - t0
        w_or = np.array([e.w for e in evs]); w_mx = evm["w"].cpu().numpy()
        sel = w_or != 0
        rel = np.abs(w_mx[sel] - w_or[sel]) / np.abs(w_or[sel])
        out["stated_err"] = {"per_event_rel_max": float(rel.max()), "per_event_rel_median": float(np.median(rel)),
                             "events": int(sel.sum()), "reference": "FP64 CPU oracle"}
        out["cpu_oracle_events_per_s"] = n_or / t_or
    except Exception as exc:                 # reported in the line, never fatal to it
        out["stated_err"] = {"error": f"{type(exc).__name__}: {exc}"}
    return out


METRIC = "gg->ttbar gg weighted events/s, FP32-mixed vs FP64 GPU at stated err; % FP peak"


def workload_config(n_events: int, dim: int, nb: int) -> dict:
    """The benchmark's workload, shared by both arms."""
    return {"workload": "gg -> t tbar g g LO, 13 TeV, 4e6 events per VEGAS iteration, mixed FP32/FP64",
            "process": "gg_ttgg", "events_per_step": n_events, "dims": dim, "bins": nb,
            "cuts": "pT(g)>30, |eta(g)|<2.5, dR(g,g)>0.4", "pdf": "synthetic 100x50 log-bicubic grid",
            "l2": "inputs far below L2; a 256 MB buffer is written between timed steps"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on this host's cores,
    a bounded sample of the same workload per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle as O
    from paper_2105_10529_gb300 import inputs as IN
    proc = IN.GG_TTGG
    phys = IN.Physics(seed=3)
    pdf = O.Pdf(IN.make_pdf_grid())
    cores = os.cpu_count() or 1
    n = max(200, 250 * cores)
    grid = O.vegas_init(IN.DIM[proc], phys.n_bins)
    for w in range(args.warmup):
        O.vegas_pass(proc, phys, pdf, grid, min(n, 64 * cores), iteration=w, n_threads=cores)
    t0 = time.perf_counter()
    for s in range(args.steps):
        r = O.vegas_pass(proc, phys, pdf, grid, n, iteration=args.warmup + s, n_threads=cores)
        grid = O.vegas_refine(r["hist"], grid, phys.alpha)
    dt = time.perf_counter() - t0
    v = n * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "events/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.events, IN.DIM[proc], phys.n_bins),
        "cpu_baseline": {"value": v, "unit": "events/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n} events per step x {args.steps} steps of the FP64 oracle (bounded sample "
                                   f"of the {args.events:.0e}-event iteration)"},
        "e2e": {"value": v, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    from paper_2105_10529_gb300 import inputs as IN
    from paper_2105_10529_gb300._lib import MF_FP64, MF_MIXED
    from paper_2105_10529_gb300.api import Context, process_info
    from paper_2105_10529_gb300.shard import allreduce_pass_sums, event_range

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    proc = IN.GG_TTGG
    if args.only_timed:
        proc = {"gg_tt": IN.GG_TT, "uu_tt": IN.UU_TT, "gg_ttg": IN.GG_TTG, "ug_ttu": IN.UG_TTU,
                "gg_ttgg": IN.GG_TTGG, "gg_ttggg": IN.GG_TTGGG}[args.process]
    phys = IN.Physics(seed=3)
    pdf = IN.make_pdf_grid()
    n_ext, dim = process_info(proc)
    nb = phys.n_bins
    N = args.events
    stream = torch.cuda.current_stream()
    ctx = Context(phys, pdf, precision=MF_MIXED, stream=stream)
    if args.sched is not None:
        ctx.set_schedule(args.sched)
    if args.hsplit is not None:
        ctx.set_helicity_split(args.hsplit)
    dev = torch.device("cuda", local)
    grid = torch.linspace(0, 1, nb + 1, dtype=torch.float64, device=dev).repeat(dim, 1).contiguous()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    from paper_2105_10529_gb300 import _lib
    import ctypes as C
    L = _lib.lib()

    def step(it, grid, n, offset, ev_it, timed_events=None):
        """One VEGAS iteration: pass over n events, (all-reduce), refine."""
        sums = torch.empty(2 + dim * nb, dtype=torch.float64, device=dev)
        if timed_events is not None:
            timed_events[0].record(stream)
        rc = L.mf_vegas_pass(ctx.ptr, proc, phys.sqrt_s, C.c_void_p(grid.data_ptr()), n, offset, ev_it, None,
                             C.c_void_p(sums.data_ptr()), None)
        if timed_events is not None:
            timed_events[1].record(stream)
        if rc:
            raise RuntimeError(L.mf_last_error(ctx.ptr))
        if world > 1:
            allreduce_pass_sums(sums, world)   # the sums of one pass over all ranks' events
        rc = L.mf_vegas_refine(ctx.ptr, dim, nb, phys.alpha, C.c_void_p(sums.data_ptr()), C.c_void_p(grid.data_ptr()))
        if rc:
            raise RuntimeError(L.mf_last_error(ctx.ptr))
        return sums

    offset, _ = event_range(N, rank)
    for w in range(args.warmup):
        step(w, grid, N, offset, w)
    torch.cuda.synchronize()
    grid_after_warmup = grid.cpu().numpy().copy()      # the e2e leg resumes from here
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    ev_pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    step_pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sums_list = []
    for s in range(args.steps):
        flush.zero_()                                  # L2 flush outside the timed step
        step_pairs[s][0].record(stream)
        sums_list.append(step(args.warmup + s, grid, N, offset, args.warmup + s, ev_pairs[s]))
        step_pairs[s][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in step_pairs]
    kern_ms = [a.elapsed_time(b) for a, b in ev_pairs]
    t_total = sum(step_ms) / 1e3
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_total = float(t.item())
    value = N * world * args.steps / t_total

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        return
    if args.only_timed:
        print(json.dumps({"only_timed": True, "process": args.process, "value": value, "unit": "events/s", "steps": args.steps,
                          "events_per_step": N, "kernel_ms": [a.elapsed_time(b) for a, b in ev_pairs]}), flush=True)
        return

    # per-step estimate of the last iteration and the pass rate
    cnt = np.zeros(2, dtype=np.uint64)
    # dominant kernel: the fused integrand (pass) -- algorithmic FLOPs per launch
    sched_eff = DEFAULT_SCHED if args.sched is None else args.sched
    fl_me = flops_per_event_me(proc, sched_eff if (args.hsplit or 1) == 1 else 2)
    fl_diagram = flops_per_event_me(proc, 3)
    # pass fraction from one extra inspection pass of the final grid
    sums_chk, evs = ctx.vegas_pass(proc, phys.sqrt_s, grid, 200_000, ev_offset=10**9, iteration=999,
                                   want_events=True, fields=("mask",))
    pass_frac = float(evs["mask"].float().mean().item())
    flops_launch = fl_me * N * pass_frac
    kern_avg_s = sum(kern_ms) / len(kern_ms) / 1e3
    achieved_tflops = flops_launch / kern_avg_s / 1e12
    pk, pk_kind = peaks()
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    # the FMA pipes' measured throughput (a microbenchmark of independent FMA chains)
    from paper_2105_10529_gb300.api import measure_fma_peak
    fma32 = measure_fma_peak(MF_MIXED, stream)
    fma64 = measure_fma_peak(MF_FP64, stream)

    # ---- FP64 GPU path on a bounded sample and the per-event error of the mixed path
    n64 = args.fp64_events
    ctx64 = Context(phys, pdf, precision=MF_FP64, stream=stream)
    ctx64.vegas_pass(proc, phys.sqrt_s, grid, 2000, iteration=0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s64, ev64 = ctx64.vegas_pass(proc, phys.sqrt_s, grid, n64, ev_offset=0, iteration=10**6,
                                 want_events=True, fields=("w", "mask"))
    e1.record(stream)
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) / 1e3
    s32, ev32 = ctx.vegas_pass(proc, phys.sqrt_s, grid, n64, ev_offset=0, iteration=10**6,
                               want_events=True, fields=("w", "mask"))
    torch.cuda.synchronize()
    w64 = ev64["w"].cpu().numpy(); w32 = ev32["w"].cpu().numpy()
    ok = (w64 != 0)
    rel64 = np.abs(w32[ok] - w64[ok]) / np.abs(w64[ok])
    sig_rel = abs(float(s32[0]) - float(s64[0])) / abs(float(s64[0]))
    err_mc = math.sqrt(max(float(s64[1]) * n64 - float(s64[0]) ** 2, 0.0) / (n64 - 1)) / abs(float(s64[0]))
    fp64_value = n64 / t64
    fp64_tflops = fl_me * n64 * float(ok.mean()) / t64 / 1e12

    # ---- stated error: the mixed path's per-event weights against the FP64 CPU oracle on a
    # subsample of the same events (same grid, Philox iteration and event numbers)
    stated = {"per_event_rel_max_vs_fp64_gpu": float(rel64.max()),
              "per_event_rel_p999_vs_fp64_gpu": float(np.quantile(rel64, 0.999)),
              "per_event_rel_median_vs_fp64_gpu": float(np.median(rel64)),
              "sigma_rel_mixed_vs_fp64_gpu": sig_rel, "mc_rel_error_of_sample": err_mc,
              "events_fp64_gpu": int(ok.sum())}
    try:
        import oracle as O
        n_or = min(args.oracle_err_events, n64)
        opdf_err = O.Pdf(pdf)
        gnp = grid.cpu().numpy()
        t0 = time.perf_counter()
        w_or = np.empty(n_or)
        for a in range(0, n_or, 20_000):
            evs_or = O.events(proc, phys, opdf_err, gnp, range(a, min(a + 20_000, n_or)), 10**6,
                              n_threads=os.cpu_count() or 1)
            w_or[a:a + len(evs_or)] = [e.w for e in evs_or]
        t_or = time.perf_counter() - t0
        sel = w_or != 0
        rel = np.abs(w32[:n_or][sel] - w_or[sel]) / np.abs(w_or[sel])
        sw_or, sw_mx = w_or.sum() / n_or, w32[:n_or].sum() / n_or
        stated.update({"per_event_rel_max": float(rel.max()), "per_event_rel_p999": float(np.quantile(rel, 0.999)),
                       "per_event_rel_median": float(np.median(rel)), "events": int(sel.sum()),
                       "sigma_rel_mixed_vs_oracle": abs(sw_mx - sw_or) / abs(sw_or),
                       "reference": f"FP64 CPU oracle, first {n_or} events of the pass ({t_or:.1f} s on "
                                    f"{os.cpu_count()} cores)"})
    except Exception as exc:                 # reported in the line, never fatal to it
        stated["oracle_error"] = f"{type(exc).__name__}: {exc}"

    # ---- end to end through the C ABI with host buffers: the timed steps again (same grid after
    # the warm-up, same Philox iterations and events) as one mf_integrate_grid call, with the PDF
    # upload from pinned host memory, the starting grid from the host and the results back
    import ctypes as C2
    pinned = torch.from_numpy(pdf).pin_memory()
    res = _lib.MfResult()
    it_host = np.zeros((args.steps, 2))
    grid_host = np.ascontiguousarray(grid_after_warmup)
    dp = C2.POINTER(C2.c_double)
    for rep in range(2):                     # the first call captures the graph, the second is timed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.mf_set_pdf(ctx.ptr, C2.cast(pinned.data_ptr(), dp))
        rc = L.mf_integrate_grid(ctx.ptr, proc, phys.sqrt_s, None, N, args.steps, args.warmup,
                                 grid_host.ctypes.data_as(dp), 0, C2.byref(res), it_host.ctypes.data_as(dp), None)
        if rc:
            raise RuntimeError(L.mf_last_error(ctx.ptr))
        t_e2e = time.perf_counter() - t0
    e2e = {"value": N * args.steps / t_e2e, "unit": "events/s",
           "h2d_bytes_per_step": int((pdf.nbytes + grid_host.nbytes) / args.steps),
           "d2h_bytes_per_step": int(it_host.nbytes / args.steps + 2 * 8 / args.steps),
           "call": f"mf_integrate_grid: {args.steps} iterations of {N} events from the grid after the warm-up, "
                   f"Philox iterations {args.warmup}..{args.warmup + args.steps - 1} (the timed steps' events)",
           "sigma_pb": res.sigma_pb}

    # ---- batched channels: the five partonic channels of p p -> t tbar + jets
    # with uneven sizes in one persistent launch per iteration (graph-replayed)
    batch = None
    if not args.no_batch:
        try:
            batch = run_batch(ctx, phys, IN, args.batch_iters)
        except Exception as exc:            # reported in the line, never fatal to it
            batch = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- the other single-process workloads (e+e-, gg -> t tbar, gg -> t tbar g)
    per_config = None
    if not args.no_configs:
        try:
            per_config = run_configs(pdf, IN, MF_FP64, MF_MIXED, stream)
        except Exception as exc:            # reported in the line, never fatal to it
            per_config = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- derivative and evaluate calls
    derivs = None
    if not args.no_configs:
        try:
            derivs = run_derivatives(ctx, phys, IN, grid, stream)
        except Exception as exc:            # reported in the line, never fatal to it
            derivs = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- g g -> t tbar g g g (the five-gluon process)
    ttggg = None
    if not args.no_configs:
        try:
            ttggg = run_ttggg(pdf, IN, MF_FP64, MF_MIXED, stream, args.ttggg_events, fma32)
        except Exception as exc:            # reported in the line, never fatal to it
            ttggg = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- helicity profile measurement and the filtered light-quark passes
    helicity = None
    if not args.no_configs:
        try:
            helicity = run_helicity(pdf, IN, MF_FP64, MF_MIXED, stream)
        except Exception as exc:            # reported in the line, never fatal to it
            helicity = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- FP64 CPU oracle on the host cores (bounded sample)
    cpu = None
    if not args.no_cpu:
        try:
            import oracle as O
            cores = os.cpu_count() or 1
            n_cpu = max(200, 1500 * cores)
            opdf = O.Pdf(pdf)
            gnp = grid.cpu().numpy()
            O.vegas_pass(proc, phys, opdf, gnp, 64, iteration=0, n_threads=cores)
            t0 = time.perf_counter()
            O.vegas_pass(proc, phys, opdf, gnp, n_cpu, iteration=7, n_threads=cores)
            dt = time.perf_counter() - t0
            cpu = {"value": n_cpu / dt, "unit": "events/s", "cores": cores, "kind": "oracle",
                   "sample": f"{n_cpu} events of one iteration at the adapted grid ({dt:.1f} s)"}
        except Exception as exc:            # reported in the line, never fatal to it
            cpu = {"error": f"{type(exc).__name__}: {exc}", "kind": "oracle"}

    line = {
        "metric": METRIC,
        "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(workload_config(N, dim, nb), colour_sum=(
            "tensor cores: tcgen05.mma kind::f16, two (128 rows x 24) x (24 x 24) per step and 256-thread CTA, "
            "bf16x2 split of "
            "the colour flows, FP32 accumulation in TMEM") if (args.sched is None or args.sched >= 2) else "FP32 FMA",
                      schedule=("one warp per event: helicity-recycled Berends-Giele currents (lanes over "
                                "current x helicity-combination tasks), five contractions per colour ordering and "
                                "configuration, amplitudes written to tensor memory"
                                if sched_eff == 4 and (args.hsplit or 1) == 1 else
                                "one warp per event, one lane per helicity of the parity-halved sum"
                                if sched_eff == 3 else f"integrand schedule {args.sched}"),
                      helicity_split=args.hsplit or 1),
        # per step: the integrand and the end-of-pass reduction (mf_vegas_pass) and the refinement
        "gpu_launches": 3 * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved_tflops / fp32_peak,
                     "traffic": ({3: DRAM_BYTES_PER_EVENT_P3, 4: DRAM_BYTES_PER_EVENT_P4}[sched_eff] * N)
                     if sched_eff in (3, 4) and (args.hsplit or 1) == 1 else None,
                     "traffic_basis": "dram__bytes_read.sum + dram__bytes_write.sum of a 1e6-event ncu capture of the "
                                      "same kernel, scaled to the launch's events",
                     "kernel": "integrand_kernel<gg_ttgg, float>",
                     "peak_basis": f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {SM_MAX_MHZ:.0f} MHz (nominal units and max clock)",
                     "flops_per_event_me": fl_me, "pass_fraction": pass_frac, "kernel_ms_avg": kern_avg_s * 1e3,
                     # context: the same events at the Feynman-diagram helicity body's count (898 kFLOP per
                     # event), i.e. the rate of diagram arithmetic this kernel replaces
                     "diagram_equivalent_tflops": fl_diagram * N * pass_frac / kern_avg_s / 1e12,
                     "diagram_equivalent_frac": fl_diagram * N * pass_frac / kern_avg_s / 1e12 / fp32_peak,
                     "measured_fma_peak_tflops": fma32, "frac_of_measured_fma_peak": achieved_tflops / fma32},
        "fp64_gpu": {"value": fp64_value, "unit": "events/s", "events": n64,
                     "achieved_tflops": fp64_tflops, "peak_nominal_tflops": FP64_PEAK_NOMINAL_TFLOPS,
                     "measured_fma_peak_tflops": fma64, "frac_of_measured_fma_peak": fp64_tflops / fma64,
                     "mixed_speedup": value / fp64_value},
        "stated_err": stated,
        "e2e": e2e,
        "clocks": clocks,
        "peaks_source": pk_kind,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if batch:
        line["batch"] = batch
    if per_config:
        line["per_config"] = per_config
    if derivs:
        line["derivatives"] = derivs
    if helicity:
        line["helicity"] = helicity
    if ttggg:
        line["gg_ttggg"] = ttggg
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_only_grad(args):
    """The derivative calls alone: d|M|^2/dp (reverse sweep) and the m_t pass of one process."""
    import torch
    from paper_2105_10529_gb300 import inputs as IN
    from paper_2105_10529_gb300.api import Context, process_info
    from paper_2105_10529_gb300._lib import MF_MIXED
    proc = {"gg_tt": IN.GG_TT, "uu_tt": IN.UU_TT, "gg_ttg": IN.GG_TTG, "ug_ttu": IN.UG_TTU,
            "gg_ttgg": IN.GG_TTGG, "gg_ttggg": IN.GG_TTGGG}[args.process]
    phys = IN.Physics(seed=3)
    _, dim = process_info(proc)
    stream = torch.cuda.current_stream()
    ctx = Context(phys, IN.make_pdf_grid(), precision=MF_MIXED, stream=stream)
    grid = torch.linspace(0, 1, phys.n_bins + 1, dtype=torch.float64, device="cuda").repeat(dim, 1).contiguous()
    n = args.events
    _, ev = ctx.vegas_pass(proc, phys.sqrt_s, grid, 4 * n, iteration=0, want_events=True, fields=("mask", "momenta"))
    mom = ev["momenta"][ev["mask"].bool()][:n].contiguous()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"only_grad": True, "process": args.process}
    for name, fn in (("evaluate_with_dme2_dp", lambda: ctx.evaluate_grad(proc, mom)),
                     ("dsigma_dmt_pass", lambda: ctx.vegas_pass_grad(proc, phys.sqrt_s, grid, n, iteration=1))):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        units = int(mom.shape[0]) if name.startswith("evaluate") else n
        out[name] = {"units": units, "per_s": units / t, "ms": t * 1e3}
    ctx.close()
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.only_grad:
        run_only_grad(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""mf_integrate's iterations run as one captured CUDA graph (replayed while the
launch parameters stay the same) and mf_integrate_grid resumes an adaptation
from a caller grid at a given Philox iteration (Sec. 2.1: the integrator's
iteration loop).  The graph must not change a result, a changed parameter
must re-capture it, and resuming must give exactly the iterations of the
pass-and-refine loop it replaces."""
import dataclasses

import numpy as np
import pytest

from paper_2105_10529_gb300 import inputs as IN
from tests.gpu_common import PHYS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdf_grid():
    return IN.make_pdf_grid()


def ctx_for(proc, prec, pdf_grid, phys=None):
    from paper_2105_10529_gb300.api import Context
    return Context(phys or PHYS[proc], pdf_grid, precision=prec)


@pytest.mark.parametrize("proc,prec,n", [(IN.EE_MUMU, 0, 100_000), (IN.GG_TTG, 1, 30_000), (IN.GG_TTGG, 1, 6000)])
def test_replay_repeats_and_recaptures(proc, prec, n, pdf_grid):
    """Replaying the captured iterations gives bit-identical results; other
    cuts, another observable or other couplings give a fresh capture whose
    result equals that of a new context."""
    phys = PHYS[proc]
    ctx = ctx_for(proc, prec, pdf_grid)
    a = ctx.integrate(proc, phys.sqrt_s, n, 3, want_grid=True)
    b = ctx.integrate(proc, phys.sqrt_s, n, 3, want_grid=True)
    assert a["sigma"] == b["sigma"] and a["error"] == b["error"] and a["n_pass"] == b["n_pass"]
    assert np.array_equal(a["grid"], b["grid"])
    if proc != IN.EE_MUMU:
        c = ctx.integrate(proc, phys.sqrt_s, n, 3, cuts=(20.0, phys.eta_max, phys.dr_min))
        assert c["n_pass"] > a["n_pass"]
        ctx.set_couplings(phys.mt + 1.0, phys.alpha_s)
        d = ctx.integrate(proc, phys.sqrt_s, n, 3)
        fresh = ctx_for(proc, prec, pdf_grid, dataclasses.replace(phys, mt=phys.mt + 1.0))
        e = fresh.integrate(proc, phys.sqrt_s, n, 3)
        fresh.close()
        assert d["sigma"] == e["sigma"] and d["n_pass"] == e["n_pass"]
        ctx.set_couplings(phys.mt, phys.alpha_s)
    ctx.set_observable(10, 0.0, 500.0)
    f = ctx.integrate(proc, phys.sqrt_s, n, 3)
    assert f["sigma"] == a["sigma"]
    h, _ = ctx.observable()
    assert abs(h.sum() / f["sigma"] - 1) < 1e-12
    ctx.set_observable(0)
    g = ctx.integrate(proc, phys.sqrt_s, n, 3)
    assert g["sigma"] == a["sigma"]
    ctx.device_status()
    ctx.close()


@pytest.mark.parametrize("proc,prec,n", [(IN.GG_TT, 0, 50_000), (IN.GG_TTGG, 1, 6000)])
def test_integrate_grid_resumes_the_pass_and_refine_loop(proc, prec, n, pdf_grid):
    """W passes with refinement (mf_vegas_pass, mf_vegas_refine) from the
    uniform grid, then K more: mf_integrate_grid from the grid after the first
    W, at Philox iterations W..W+K-1, gives the same per-iteration estimates,
    the same final grid, and from the uniform grid at iteration 0 exactly
    mf_integrate."""
    phys = PHYS[proc]
    ctx = ctx_for(proc, prec, pdf_grid)
    dim = IN.DIM[proc]
    nb = phys.n_bins
    grid = torch.linspace(0, 1, nb + 1, dtype=torch.float64, device="cuda").repeat(dim, 1).contiguous()
    W, K = 2, 3
    per = []
    g_w = None
    for it in range(W + K):
        if it == W:
            g_w = grid.cpu().numpy().copy()
        sums, _ = ctx.vegas_pass(proc, phys.sqrt_s, grid, n, iteration=it)
        s = sums.cpu().numpy()
        per.append((s[0], (n * s[1] - s[0] ** 2) / (n - 1)))
        if it < W + K - 1:
            from paper_2105_10529_gb300 import _lib
            import ctypes as C
            assert _lib.lib().mf_vegas_refine(ctx.ptr, dim, nb, phys.alpha, C.c_void_p(sums.data_ptr()),
                                              C.c_void_p(grid.data_ptr())) == 0
    torch.cuda.synchronize()
    r = ctx.integrate_grid(proc, phys.sqrt_s, n, K, g_w, first_iteration=W)
    ref = np.array(per[W:])
    assert np.allclose(r["per_iter"], ref, rtol=1e-13, atol=0)
    assert np.array_equal(r["grid"], grid.cpu().numpy())
    u = (np.arange(nb + 1) / nb)[None, :].repeat(dim, 0)    # the uniform grid as the library forms it, i / n_bins
    a = ctx.integrate_grid(proc, phys.sqrt_s, n, K, u, first_iteration=0)
    b = ctx.integrate(proc, phys.sqrt_s, n, K, want_grid=True)
    assert a["sigma"] == b["sigma"] and np.array_equal(a["grid"], b["grid"])
    from paper_2105_10529_gb300._lib import MfError
    import ctypes as C
    from paper_2105_10529_gb300 import _lib
    res = _lib.MfResult()
    assert _lib.lib().mf_integrate_grid(ctx.ptr, proc, phys.sqrt_s, None, n, 2, 0, None, 0, C.byref(res),
                                        None, None) == 1
    ctx.close()


def test_graphs_of_several_channels_are_kept(pdf_grid):
    """Channels integrated in turn on one context each replay their own graph:
    every result equals the first call's, also after more parameter sets than
    the context keeps (the evicted one is captured afresh)."""
    phys = PHYS[IN.GG_TT]
    ctx = ctx_for(IN.GG_TT, 1, pdf_grid)
    runs = [(IN.GG_TT, 20_000), (IN.UU_TT, 20_000), (IN.GG_TTG, 10_000), (IN.GG_TTGG, 3000)]
    first = {r: ctx.integrate(r[0], phys.sqrt_s, r[1], 3, want_grid=True) for r in runs}
    for _ in range(2):
        for r in runs:
            x = ctx.integrate(r[0], phys.sqrt_s, r[1], 3, want_grid=True)
            assert x["sigma"] == first[r]["sigma"] and np.array_equal(x["grid"], first[r]["grid"]), r
    # 20 more parameter sets push the first ones out
    for k in range(20):
        ctx.integrate(IN.GG_TT, phys.sqrt_s, 1000 + k, 1)
    for r in runs:
        x = ctx.integrate(r[0], phys.sqrt_s, r[1], 3, want_grid=True)
        assert x["sigma"] == first[r]["sigma"] and np.array_equal(x["grid"], first[r]["grid"]), r
    ctx.close()

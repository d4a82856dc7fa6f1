"""mf_vegas_pass_static: the pass entry point for callers that cannot
allocate GPU memory (their host owns every device buffer, or they must not
let a call synchronise the device the way cudaMalloc may).  It keeps its
scratch in a fixed array inside the library.  Its sums must match those of
the context-based mf_vegas_pass on the same inputs, call after call: the
array keeps the previous call's contents, so a second call checks that
nothing stale leaks into the result.  This file is collected last."""
import ctypes as C

import numpy as np
import pytest

from paper_2105_10529_gb300 import inputs as IN

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _static_pass(L, cfg, proc, phys, pdf_t, grid_t, n, offset, iteration, sums_t):
    nf, nx, nq = pdf_t.shape
    return L.mf_vegas_pass_static(proc, C.byref(cfg), phys.sqrt_s, C.c_void_p(pdf_t.data_ptr()), nf, nx, nq,
                                  IN.PDF_X_MIN, IN.PDF_Q2_MIN, IN.PDF_Q2_MAX, C.c_void_p(grid_t.data_ptr()), n, offset,
                                  iteration, C.c_void_p(sums_t.data_ptr()),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("proc,prec", [(IN.GG_TTGG, 1), (IN.GG_TT, 0)])
def test_static_scratch_pass_matches_context_pass(proc, prec):
    from paper_2105_10529_gb300 import _lib
    from paper_2105_10529_gb300.api import Context, make_config, process_info
    from tests.gpu_common import PHYS, random_grid
    L = _lib.lib()
    phys = PHYS[proc]
    _, dim = process_info(proc)
    pdf = IN.make_pdf_grid()
    pdf_t = torch.tensor(pdf, device="cuda")
    cfg = make_config(phys, prec)
    ctx = Context(phys, pdf, precision=prec)
    ctx.set_schedule(0)     # the allocation-free pass runs schedule 0 (one event per thread)
    n = 20_000 if proc == IN.GG_TTGG else 200_000
    for call, (seed, offset, it) in enumerate([(proc, 0, 2), (proc + 10, 12345, 5)]):
        grid_t = torch.tensor(random_grid(dim, seed=seed), device="cuda")
        ref, _ = ctx.vegas_pass(proc, phys.sqrt_s, grid_t, n, ev_offset=offset, iteration=it)
        out = torch.full((2 + dim * phys.n_bins,), float("nan"), dtype=torch.float64, device="cuda")
        rc = _static_pass(L, cfg, proc, phys, pdf_t, grid_t, n, offset, it, out)
        assert rc == 0, rc
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a)), f"call {call}"
        # same kernels and per-event values; only the CTA count, hence the summation order, may differ
        tol = 1e-12 if prec == 0 else 1e-6
        assert np.allclose(a, b, rtol=tol, atol=1e-300), (call, np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))
    ctx.close()


def test_static_scratch_pass_rejects_bad_sizes():
    from paper_2105_10529_gb300 import _lib
    from paper_2105_10529_gb300.api import make_config
    L = _lib.lib()
    phys = IN.Physics(seed=3)
    pdf_t = torch.tensor(IN.make_pdf_grid(), device="cuda")
    grid_t = torch.zeros((18, 51), dtype=torch.float64, device="cuda")
    out = torch.zeros(2 + 18 * 50, dtype=torch.float64, device="cuda")
    cfg = make_config(phys, 1)
    cfg.n_bins = 65                                     # above the 64-bin maximum
    assert _static_pass(L, cfg, IN.GG_TTGG, phys, pdf_t, grid_t, 100, 0, 0, out) == 1
    cfg = make_config(phys, 1)
    assert _static_pass(L, cfg, IN.GG_TTGG, phys, pdf_t, grid_t, 0, 0, 0, out) == 1   # no events
    assert _static_pass(L, cfg, 17, phys, pdf_t, grid_t, 100, 0, 0, out) == 1         # unknown process


@pytest.mark.parametrize("proc,prec", [(IN.GG_TTGG, 1), (IN.GG_TTG, 0)])
def test_static_pass_leaves_context_observable_working(proc, prec):
    """A call of the allocation-free pass must not lower the shared-memory
    limit of the process's kernels below what a context's passes with the
    p_T histogram need: a context created before it still integrates with the
    histogram on, and gives the same result as before the call."""
    from paper_2105_10529_gb300 import _lib
    from paper_2105_10529_gb300.api import Context, make_config, process_info
    from tests.gpu_common import PHYS, random_grid
    L = _lib.lib()
    phys = PHYS[proc]
    _, dim = process_info(proc)
    pdf = IN.make_pdf_grid()
    ctx = Context(phys, pdf, precision=prec)
    ctx.set_observable(20, 0.0, 800.0)
    before = ctx.integrate(proc, phys.sqrt_s, 4000, 2)
    h_before = ctx.observable()[0]
    pdf_t = torch.tensor(pdf, device="cuda")
    grid_t = torch.tensor(random_grid(dim, seed=77), device="cuda")
    out = torch.zeros(2 + dim * phys.n_bins, dtype=torch.float64, device="cuda")
    assert _static_pass(L, make_config(phys, prec), proc, phys, pdf_t, grid_t, 3000, 0, 1, out) == 0
    torch.cuda.synchronize()
    after = ctx.integrate(proc, phys.sqrt_s, 4000, 2)
    ctx.device_status()
    assert after["status"] == 0
    assert after["sigma"] == before["sigma"]
    assert np.array_equal(ctx.observable()[0], h_before)
    ctx.close()

"""Derivatives on the GPU: d sigma/d alpha_s exact, d sigma/d m_t against
central finite differences (GPU and oracle, frozen masks, h = 1e-3 m_t),
mixed against FP64, d|M|^2/dp against finite differences and Lorentz
invariance, the gg -> t tbar pathwise derivative against the derivative of a
deterministic quadrature, and the torch.autograd wrappers."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from tests.gpu_common import PHYS, random_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K_AS = {IN.GG_TT: 2, IN.GG_TTG: 3, IN.GG_TTGG: 4, IN.GG_TTGGG: 5}


@pytest.fixture(scope="module")
def pdf_grid():
    return IN.make_pdf_grid()


def ctx_for(proc, prec, pdf_grid):
    from paper_2105_10529_gb300.api import Context
    return Context(PHYS.get(proc, IN.Physics(seed=6)), pdf_grid, precision=prec)


def gpu_fd(ctx, proc, phys, grid, n, mask, h, it):
    vals = []
    for m in (phys.mt + h, phys.mt - h):
        ctx.set_couplings(m, phys.alpha_s)
        s, _ = ctx.vegas_pass(proc, phys.sqrt_s, grid, n, iteration=it, mask_in=mask)
        vals.append(float(s[0]))
    ctx.set_couplings(phys.mt, phys.alpha_s)
    return (vals[0] - vals[1]) / (2 * h)


@pytest.mark.parametrize("proc,prec", [(IN.GG_TT, 0), (IN.GG_TTG, 0), (IN.GG_TT, 1), (IN.GG_TTG, 1), (IN.GG_TTGG, 0),
                                       (IN.GG_TTGG, 1), (IN.GG_TTGGG, 0), (IN.GG_TTGGG, 1)])
def test_mt_and_alphas_derivatives(proc, prec, pdf_grid):
    phys = PHYS.get(proc, IN.Physics(seed=6))
    grid = torch.tensor(random_grid(IN.DIM[proc], seed=20 + proc), device="cuda")
    n = {IN.GG_TT: 20000, IN.GG_TTG: 4000, IN.GG_TTGG: 1000, IN.GG_TTGGG: 300}[proc]
    it = 6
    ctx = ctx_for(proc, prec, pdf_grid)
    d = ctx.vegas_pass_grad(proc, phys.sqrt_s, grid, n, iteration=it).cpu().numpy()
    base, ev = ctx.vegas_pass(proc, phys.sqrt_s, grid, n, iteration=it, want_events=True, fields=("mask",))
    # the derivative pass reproduces the value of the pass
    assert abs(d[0] / float(base[0]) - 1) < (1e-12 if prec == 0 else 1e-5)
    # d sigma / d alpha_s = k sigma / alpha_s exactly
    assert abs(d[3] - K_AS[proc] * d[0] / phys.alpha_s) <= 1e-12 * abs(d[3])
    # d sigma / d m_t against central differences of the FP64 value pass with frozen masks
    ctx64 = ctx_for(proc, 0, pdf_grid)
    fd = gpu_fd(ctx64, proc, phys, grid, n, ev["mask"], 1e-3 * phys.mt, it)
    assert abs(d[1] - fd) < 1e-4 * abs(fd), (d[1], fd)
    ctx.close(); ctx64.close()


@pytest.mark.parametrize("proc", [IN.GG_TT, IN.GG_TTG, IN.GG_TTGG, IN.GG_TTGGG])
def test_mt_derivative_matches_oracle_fd(proc, pdf_grid):
    """The FP64 derivative pass (forward tangents for g g -> t tbar (g), the
    reverse sweep for g g -> t tbar g g (g)) against central differences of the
    oracle's pass with the masks frozen, to 1e-4."""
    phys = PHYS.get(proc, IN.Physics(seed=6))
    gnp = random_grid(IN.DIM[proc], seed=30 + proc)
    grid = torch.tensor(gnp, device="cuda")
    n = {IN.GG_TT: 3000, IN.GG_TTG: 600, IN.GG_TTGG: 200, IN.GG_TTGGG: 48}[proc]
    it = 2
    ctx = ctx_for(proc, 0, pdf_grid)
    d = ctx.vegas_pass_grad(proc, phys.sqrt_s, grid, n, iteration=it).cpu().numpy()
    opdf = O.Pdf(pdf_grid)
    base = O.vegas_pass(proc, phys, opdf, gnp, n, iteration=it, want_mask=True)
    h = 1e-3 * phys.mt
    hi = O.vegas_pass(proc, IN.Physics(**{**phys.as_dict(), "mt": phys.mt + h}), opdf, gnp, n, it, mask_in=base["mask"])
    lo = O.vegas_pass(proc, IN.Physics(**{**phys.as_dict(), "mt": phys.mt - h}), opdf, gnp, n, it, mask_in=base["mask"])
    fd = (hi["sum_w"] - lo["sum_w"]) / (2 * h)
    assert abs(d[1] - fd) < 1e-4 * abs(fd), (d[1], fd)
    ctx.close()


@pytest.mark.parametrize("proc", [IN.GG_TT, IN.GG_TTG, IN.GG_TTGG, IN.GG_TTGGG])
def test_mixed_derivative_matches_fp64(proc, pdf_grid):
    phys = PHYS.get(proc, IN.Physics(seed=6))
    grid = torch.tensor(random_grid(IN.DIM[proc], seed=40 + proc), device="cuda")
    n = {IN.GG_TTGG: 4000, IN.GG_TTGGG: 1000}.get(proc, 20000)
    a = ctx_for(proc, 0, pdf_grid).vegas_pass_grad(proc, phys.sqrt_s, grid, n, iteration=3).cpu().numpy()
    b = ctx_for(proc, 1, pdf_grid).vegas_pass_grad(proc, phys.sqrt_s, grid, n, iteration=3).cpu().numpy()
    assert abs(b[1] / a[1] - 1) < 1e-5


def boost_direction(p):
    """Infinitesimal boost along z of every momentum: dE = p_z, dp_z = E."""
    d = np.zeros_like(p)
    d[..., 0] = p[..., 3]
    d[..., 3] = p[..., 0]
    return d


def rotation_direction(p):
    """Infinitesimal rotation about z of every momentum: dp_x = -p_y, dp_y = p_x."""
    d = np.zeros_like(p)
    d[..., 1] = -p[..., 2]
    d[..., 2] = p[..., 1]
    return d


def boost_x_direction(p):
    """Infinitesimal boost along x: dE = p_x, dp_x = E."""
    d = np.zeros_like(p)
    d[..., 0] = p[..., 1]
    d[..., 1] = p[..., 0]
    return d


@pytest.mark.parametrize("proc,prec", [(IN.GG_TT, 0), (IN.GG_TTG, 0), (IN.GG_TTGG, 0), (IN.GG_TTGG, 1),
                                       (IN.GG_TTGGG, 0), (IN.GG_TTGGG, 1), (IN.UG_TTU, 1)])
def test_evaluate_gradient(proc, prec, pdf_grid):
    """d|M|^2/dp of mf_evaluate (the reverse sweep of the Berends-Giele recursion
    for the gluon processes, forward tangents for u g -> t tbar u): every
    component against fourth-order differences of the same formula (the value
    the derivative call returns, in FP64), the value itself against mf_evaluate
    (the same |M|^2 on shell), and zero along the Lorentz generators (two boosts,
    one rotation), the directions in which |M|^2 does not change."""
    phys = PHYS[proc]
    rng = np.random.default_rng(50 + proc)
    n_ext = IN.N_EXT[proc]
    nf = n_ext - 2
    moms = []
    for rs in (800.0, 2500.0):
        for _ in range(3):
            pf, _ = O.rambo(nf, rs, [phys.mt, phys.mt] + [0.0] * (nf - 2), rng.random(4 * nf))
            moms.append(np.vstack([[[rs / 2, 0, 0, rs / 2], [rs / 2, 0, 0, -rs / 2]], pf]))
    P = np.array(moms)
    ctx = ctx_for(proc, prec, pdf_grid)
    ctx64 = ctx_for(proc, 0, pdf_grid)
    me, g = ctx.evaluate_grad(proc, torch.tensor(P, device="cuda"))
    me, g = me.cpu().numpy(), g.cpu().numpy()
    plain = ctx64.evaluate(proc, torch.tensor(P, device="cuda")).cpu().numpy()
    assert np.all(np.abs(me - plain) <= (1e-11 if prec == 0 else 1e-5) * np.abs(plain)), (me, plain)
    for e in range(len(P)):
        for (i, c) in [(2, 0), (2, 3), (3, 1), (0, 0), (1, 3), (n_ext - 1, 2)]:
            # fourth-order central differences (error O(h^4)) of the FP64 value of the same formula
            # at h and h / 2; their disagreement estimates the difference's own error (rounding of
            # the values grows as 1/h, truncation falls as h^4), which widens the FP64 tolerance
            # at points where the many-gluon value carries rounding of its own
            fds = []
            for h in (1e-4 * abs(P[e, i, 0]), 0.5e-4 * abs(P[e, i, 0])):
                q = np.repeat(P[e:e + 1], 4, axis=0)
                for r, k in enumerate((2, 1, -1, -2)):
                    q[r, i, c] += k * h
                v = ctx64.evaluate_grad(proc, torch.tensor(q, device="cuda"))[0].cpu().numpy()
                fds.append((-v[0] + 8 * v[1] - 8 * v[2] + v[3]) / (12 * h))
            fd, fd_err = fds[1], 3.0 * abs(fds[0] - fds[1])
            scale = np.abs(g[e]).max() * abs(P[e, i, 0])
            tol = (1e-7 if prec == 0 else 3e-5) * scale + fd_err * abs(P[e, i, 0])
            assert fd_err < 1e-4 * np.abs(g[e]).max(), (e, i, c, fds)
            assert abs(g[e, i, c] - fd) * abs(P[e, i, 0]) < tol, (e, i, c, g[e, i, c], fds)
        # |M|^2 is Lorentz invariant: no derivative along the boost and rotation generators
        for gen in (boost_direction, boost_x_direction, rotation_direction):
            d = gen(P[e])
            along = float(np.sum(g[e] * d))
            assert abs(along) < (1e-9 if prec == 0 else 1e-4) * float(np.sum(np.abs(g[e] * d))), (gen.__name__, along)
    ctx.close(); ctx64.close()


@pytest.mark.parametrize("proc", [IN.GG_TT, IN.GG_TTG, IN.GG_TTGG, IN.GG_TTGGG])
def test_mixed_evaluate_gradient_matches_fp64(proc, pdf_grid):
    """The mixed-precision reverse sweep against the FP64 one: every component of
    d|M|^2/dp within 1e-5 of the event's largest component."""
    phys = PHYS[proc]
    rng = np.random.default_rng(70 + proc)
    nf = IN.N_EXT[proc] - 2
    moms = []
    for rs in (600.0, 1500.0, 4000.0):
        for _ in range(4):
            pf, _ = O.rambo(nf, rs, [phys.mt, phys.mt] + [0.0] * (nf - 2), rng.random(4 * nf))
            moms.append(np.vstack([[[rs / 2, 0, 0, rs / 2], [rs / 2, 0, 0, -rs / 2]], pf]))
    P = torch.tensor(np.array(moms), device="cuda")
    _, g64 = ctx_for(proc, 0, pdf_grid).evaluate_grad(proc, P)
    _, g32 = ctx_for(proc, 1, pdf_grid).evaluate_grad(proc, P)
    g64, g32 = g64.cpu().numpy(), g32.cpu().numpy()
    for e in range(len(moms)):
        scale = np.abs(g64[e]).max()
        assert np.abs(g32[e] - g64[e]).max() <= 1e-5 * scale, (e, float(np.abs(g32[e] - g64[e]).max() / scale))


def test_gg_tt_pathwise_derivative_matches_quadrature(pdf_grid):
    """Without cuts the pathwise derivative is unbiased for d sigma/d m_t:
    compare with the m_t derivative of a deterministic quadrature."""
    from tests.test_oracle_integration import sigma_hadronic_quadrature, sig_hat_gg
    proc = IN.GG_TT
    phys = PHYS[proc]
    opdf = O.Pdf(pdf_grid)
    h = 1e-3 * phys.mt
    q = [sigma_hadronic_quadrature(IN.Physics(**{**phys.as_dict(), "mt": m}), opdf,
                                   sig_hat_gg(IN.Physics(**{**phys.as_dict(), "mt": m})), 0, 0, n=96)
         for m in (phys.mt + h, phys.mt - h)]
    dq = (q[0] - q[1]) / (2 * h)
    ctx = ctx_for(proc, 0, pdf_grid)
    grid = torch.tensor(O.vegas_init(IN.DIM[proc]), device="cuda")
    n = 4_000_000
    d = ctx.vegas_pass_grad(proc, phys.sqrt_s, grid, n, iteration=0).cpu().numpy()
    err = math.sqrt(max(d[2] * n - d[1] ** 2, 0.0) / (n - 1))
    assert abs(d[1] - dq) < 4 * err, (d[1], dq, err)
    ctx.close()


def test_autograd_wrappers(pdf_grid):
    from paper_2105_10529_gb300.autograd import cross_section, matrix_element
    proc = IN.GG_TTG
    phys = PHYS[proc]
    ctx = ctx_for(proc, 0, pdf_grid)
    grid = torch.tensor(random_grid(IN.DIM[proc], seed=60), device="cuda")
    mt = torch.tensor(phys.mt, dtype=torch.float64, requires_grad=True)
    a_s = torch.tensor(phys.alpha_s, dtype=torch.float64, requires_grad=True)
    sig = cross_section(mt, a_s, ctx, proc, phys.sqrt_s, grid, 3000, iteration=1)
    sig.backward()
    d = ctx.vegas_pass_grad(proc, phys.sqrt_s, grid, 3000, iteration=1).cpu().numpy()
    assert abs(sig.item() - d[0]) <= 1e-12 * abs(d[0])
    assert abs(mt.grad.item() - d[1]) <= 1e-12 * abs(d[1])
    assert abs(a_s.grad.item() - d[3]) <= 1e-12 * abs(d[3])
    rng = np.random.default_rng(61)
    pf, _ = O.rambo(3, 1500.0, [phys.mt, phys.mt, 0.0], rng.random(12))
    P = torch.tensor(np.vstack([[[750.0, 0, 0, 750.0], [750.0, 0, 0, -750.0]], pf])[None], device="cuda",
                     requires_grad=True)
    m2 = matrix_element(P, ctx, proc)
    m2.sum().backward()
    _, g = ctx.evaluate_grad(proc, P.detach())
    assert torch.allclose(P.grad, g, rtol=1e-14, atol=0)
    ctx.close()


@pytest.mark.parametrize("proc,prec", [(IN.GG_TT, 0), (IN.UG_TTU, 1), (IN.GG_TTGG, 1)])
def test_integrate_want_grads(proc, prec, pdf_grid):
    """mf_integrate with want_grads: the derivative fields are the derivative
    pass at the returned final grid on Philox iteration n_iter."""
    phys = PHYS[proc]
    ctx = ctx_for(proc, prec, pdf_grid)
    n, n_iter = 4000, 2
    r = ctx.integrate(proc, phys.sqrt_s, n, n_iter, want_grid=True, want_grads=True)
    g = ctx.vegas_pass_grad(proc, phys.sqrt_s, torch.tensor(r["grid"], device="cuda"), n,
                            iteration=n_iter).cpu().numpy()
    assert r["dsigma_dmt"] == g[1] and r["dsigma_dalphas"] == g[3]
    var = (n * g[2] - g[1] ** 2) / (n - 1)
    assert r["dsigma_dmt_error"] == pytest.approx(math.sqrt(var), rel=1e-12)
    assert r["dsigma_dmt"] < 0.0 < r["dsigma_dalphas"]
    plain = ctx.integrate(proc, phys.sqrt_s, n, n_iter)
    assert plain["sigma"] == r["sigma"] and plain["dsigma_dmt"] == 0.0
    ctx.close()

"""The double-float arithmetic of the mixed-precision kinematics (mf_selftest_df) against the
GPU's FP64 functions at the same points: each argument is first rounded to the nearest
double-float, so that the comparison measures the function and not the rounding of its
input.  Bounds: a few 1e-14 relative from the double-word error analyses (sums 3u^2,
products 4u^2, quotients 15u^2, u = 2^-24) and the truncated series, with margin."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _df_round(x: np.ndarray) -> np.ndarray:
    """The nearest double-float of each double, as a double (hi + lo)."""
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi.astype(np.float64) + lo.astype(np.float64)


def _run(fn, x):
    from paper_2105_10529_gb300.api import selftest_df
    xr = _df_round(np.asarray(x, dtype=np.float64))
    xt = torch.tensor(xr, dtype=torch.float64, device="cuda")
    y = selftest_df(fn, xt)
    torch.cuda.synchronize()
    return xt, y


def _rel(y, ref):
    return ((y - ref).abs() / ref.abs().clamp_min(1e-300)).max().item()


def test_exp():
    rng = np.random.default_rng(11)
    # down to e^-60: below about 2e-31 a double-float's tail is subnormal and its relative
    # precision falls towards float's (the exponent range is float's)
    x = np.concatenate([rng.uniform(-20.0, 5.0, 200_000), rng.uniform(-60.0, 87.0, 20_000),
                        np.linspace(-1e-3, 1e-3, 2001), np.array([0.0, 0.5 * math.log(2.0), -0.5 * math.log(2.0)])])
    xt, y = _run("exp", x)
    assert _rel(y, torch.exp(xt)) < 2e-13


def test_log():
    rng = np.random.default_rng(12)
    x = np.concatenate([10.0 ** rng.uniform(-17.0, 9.0, 200_000), 1.0 + rng.uniform(-1e-6, 1e-6, 20_000),
                        rng.uniform(0.5, 2.0, 20_000), np.array([1.0, 2.0, 0.5, 1e-16])])
    xt, y = _run("log", x)
    ref = torch.log(xt)
    err = ((y - ref).abs() / ref.abs().clamp_min(1.0)).max().item()
    assert err < 2e-13
    _, y0 = _run("log", np.array([0.0]))
    assert y0.item() == -math.inf


def test_sqrt():
    rng = np.random.default_rng(13)
    x = np.concatenate([10.0 ** rng.uniform(-20.0, 20.0, 200_000), np.array([1.0, 4.0, 2.0])])
    xt, y = _run("sqrt", x)
    assert _rel(y, torch.sqrt(xt)) < 1e-13
    _, y0 = _run("sqrt", np.array([0.0]))
    assert y0.item() == 0.0


@pytest.mark.parametrize("fn", ["sinpi", "cospi"])
def test_sincospi(fn):
    rng = np.random.default_rng(14)
    quad = np.repeat(np.arange(0, 9) * 0.25, 2001) + np.tile(np.linspace(-1e-6, 1e-6, 2001), 9)
    x = np.concatenate([rng.uniform(0.0, 2.0, 200_000), rng.uniform(-4.0, 4.0, 20_000), quad])
    xt, y = _run(fn, x)
    # the reference reduces first, so that pi x is not rounded at large x: x = n/2 + r
    n = torch.round(2.0 * xt)
    r = xt - 0.5 * n
    t = math.pi * r
    q = n.remainder(4)
    s, c = torch.sin(t), torch.cos(t)
    if fn == "sinpi":
        ref = torch.where(q == 0, s, torch.where(q == 1, c, torch.where(q == 2, -s, -c)))
    else:
        ref = torch.where(q == 0, c, torch.where(q == 1, -s, torch.where(q == 2, -c, s)))
    assert (y - ref).abs().max().item() < 1e-13


def test_recip_and_square():
    rng = np.random.default_rng(15)
    x = np.concatenate([10.0 ** rng.uniform(-15.0, 15.0, 200_000) * np.sign(rng.uniform(-1, 1, 200_000))])
    xt, y = _run("recip", x)
    assert _rel(y, 1.0 / xt) < 1e-13
    xs = x[np.abs(x) < 1e15]
    xt, y = _run("square", xs)
    assert _rel(y, xt * xt) < 1e-13


def test_arguments():
    from paper_2105_10529_gb300 import _lib
    L = _lib.lib()
    assert L.mf_selftest_df(7, None, 0, None, None) == 1   # MF_ERR_ARG
    assert L.mf_selftest_df(-1, None, 0, None, None) == 1   # MF_ERR_ARG
    assert L.mf_selftest_df(0, None, -1, None, None) == 1   # MF_ERR_ARG
    assert L.mf_selftest_df(0, None, 5, None, None) == 1   # MF_ERR_ARG
    assert L.mf_selftest_df(0, None, 0, None, None) == 0

"""Python access to the FP64 CPU oracle (plain C, ``oracle/*.c``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the CUDA path never does.
The oracle shares no code with the CUDA path; both take their inputs from
``paper_2105_10529_gb300.inputs``.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None


class OrParams(C.Structure):
    _fields_ = [("sqrt_s", C.c_double), ("mt", C.c_double), ("alpha_s", C.c_double),
                ("mz", C.c_double), ("wz", C.c_double), ("alpha_em_inv", C.c_double),
                ("gf", C.c_double), ("pt_min", C.c_double), ("eta_max", C.c_double),
                ("dr_min", C.c_double), ("seed", C.c_uint64), ("channel", C.c_uint32),
                ("n_bins", C.c_int), ("alpha", C.c_double)]


class OrPdf(C.Structure):
    _fields_ = [("xf", C.POINTER(C.c_double)), ("n_flav", C.c_int), ("nx", C.c_int), ("nq", C.c_int),
                ("x_min", C.c_double), ("q2_min", C.c_double), ("q2_max", C.c_double)]


class OrEvent(C.Structure):
    _fields_ = [("u", C.c_double * 32), ("x", C.c_double * 32), ("bins", C.c_uint8 * 32),
                ("jac_vegas", C.c_double), ("x1", C.c_double), ("x2", C.c_double),
                ("shat", C.c_double), ("jac_parton", C.c_double), ("w_ps", C.c_double),
                ("p", C.c_double * 28), ("plab", C.c_double * 28), ("mask", C.c_int),
                ("muf2", C.c_double), ("f1", C.c_double), ("f2", C.c_double),
                ("me2", C.c_double), ("w", C.c_double)]


class OrResult(C.Structure):
    _fields_ = [("sigma", C.c_double), ("error", C.c_double), ("chi2dof", C.c_double),
                ("n_pass", C.c_int64)]


class OrProcInfo(C.Structure):
    _fields_ = [("n_ext", C.c_int), ("n_final", C.c_int), ("dim", C.c_int), ("n_hel", C.c_int),
                ("as_power", C.c_int), ("avg", C.c_double), ("sym", C.c_double)]


_D = C.POINTER(C.c_double)
_U8 = C.POINTER(C.c_uint8)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "or_philox4x32_10": (None, [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
            "or_u01": (C.c_double, [C.c_uint32, C.c_uint32]),
            "or_uniforms": (None, [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, _D]),
            "or_vegas_init": (None, [_D, C.c_int, C.c_int]),
            "or_vegas_map": (C.c_double, [_D, C.c_int, C.c_int, _D, _D, _U8]),
            "or_vegas_refine": (None, [_D, _D, C.c_int, C.c_int, C.c_double]),
            "or_vegas_combine": (None, [C.c_int, _D, _D, _D, _D, _D]),
            "or_parton_map": (None, [C.c_double, C.c_double, C.c_double, _D, _D, _D]),
            "or_rambo": (C.c_int, [C.c_int, C.c_double, _D, _D, _D, _D]),
            "or_rambo_massless_volume": (C.c_double, [C.c_int, C.c_double]),
            "or_cuts": (C.c_int, [C.c_int, C.POINTER(OrParams), _D]),
            "or_muf2": (C.c_double, [C.c_int, C.POINTER(OrParams), _D]),
            "or_pdf_xf": (C.c_double, [C.POINTER(OrPdf), C.c_int, C.c_double, C.c_double]),
            "or_me2": (C.c_double, [C.c_int, C.POINTER(OrParams), _D]),
            "or_me2_ee_mumu_closed": (C.c_double, [C.POINTER(OrParams), _D]),
            "or_me2_gg_tt_closed": (C.c_double, [C.c_double, C.c_double, _D]),
            "or_me2_uu_tt_closed": (C.c_double, [C.c_double, C.c_double, _D]),
            "or_me2_uu_tt_diagram": (C.c_double, [C.c_double, C.c_double, _D]),
            "or_me2_ug_ttu": (C.c_double, [C.c_double, C.c_double, _D]),
            "or_amp2_ug_ttu_ward": (C.c_double, [C.c_double, C.c_double, _D]),
            "or_bg_partial": (None, [C.c_int, _D, _D, _D, _D, C.c_double, C.c_double, C.c_int, C.c_int, _I, _D]),
            "or_me2_bg": (C.c_double, [C.c_int, _D, C.c_int, C.c_double, C.c_double]),
            "or_colour_matrix": (None, [C.c_int, _D]),
            "or_gellmann_T": (None, [C.c_int, _D]),
            "or_proc_info_get": (C.c_int, [C.c_int, C.POINTER(OrProcInfo)]),
            "or_event": (C.c_int, [C.c_int, C.POINTER(OrParams), C.POINTER(OrPdf), _D, C.c_uint64,
                                   C.c_uint32, _I, C.POINTER(OrEvent)]),
            "or_events": (C.c_int, [C.c_int, C.POINTER(OrParams), C.POINTER(OrPdf), _D, C.POINTER(C.c_uint64),
                                    C.c_int64, C.c_uint32, C.POINTER(OrEvent), C.c_int]),
            "or_pass": (C.c_int, [C.c_int, C.POINTER(OrParams), C.POINTER(OrPdf), _D, C.c_int64, C.c_uint32,
                                  _U8, _U8, _D, _D, _D, C.POINTER(C.c_int64), C.c_int]),
            "or_integrate": (C.c_int, [C.c_int, C.POINTER(OrParams), C.POINTER(OrPdf), C.c_int64, C.c_int,
                                       _D, _D, C.POINTER(OrResult), C.c_int]),
            "or_obs_bin": (C.c_int, [C.c_double, C.c_double, C.c_int, C.c_double, C.c_double]),
            "or_pass_obs": (C.c_int, [C.c_int, C.POINTER(OrParams), C.POINTER(OrPdf), _D, C.c_int64, C.c_uint32,
                                      C.c_int, C.c_double, C.c_double, _D, _D, _D, C.c_int]),
            "or_integrate_obs": (C.c_int, [C.c_int, C.POINTER(OrParams), C.POINTER(OrPdf), C.c_int64, C.c_int,
                                           C.c_int, C.c_double, C.c_double, _D, _D, _D, C.POINTER(OrResult),
                                           C.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def params(phys) -> OrParams:
    """OrParams from an ``inputs.Physics`` (or any object with the same fields)."""
    d = phys.as_dict() if hasattr(phys, "as_dict") else dict(phys)
    return OrParams(**{k: d[k] for k, _ in OrParams._fields_})


class Pdf:
    """Keeps the grid array alive alongside its C view."""

    def __init__(self, grid: np.ndarray, x_min=1e-6, q2_min=1.0, q2_max=1e8):
        self.grid = _f64(grid)
        nf, nx, nq = self.grid.shape
        self.c = OrPdf(_dp(self.grid), nf, nx, nq, x_min, q2_min, q2_max)

    def xf(self, flav: int, x: float, q2: float) -> float:
        return lib().or_pdf_xf(C.byref(self.c), flav, x, q2)


def proc_info(proc: int) -> OrProcInfo:
    o = OrProcInfo()
    if lib().or_proc_info_get(proc, C.byref(o)):
        raise ValueError(proc)
    return o


def philox(ctr, key) -> tuple:
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return tuple(o)


def u01(a: int, b: int) -> float:
    return lib().or_u01(a, b)


def uniforms(seed: int, event: int, iteration: int, channel: int, dim: int) -> np.ndarray:
    u = np.zeros(dim)
    lib().or_uniforms(seed, event, iteration, channel, dim, _dp(u))
    return u


def vegas_init(dim: int, nb: int = 50) -> np.ndarray:
    g = np.zeros((dim, nb + 1))
    lib().or_vegas_init(_dp(g), dim, nb)
    return g


def vegas_map(grid: np.ndarray, u: np.ndarray):
    grid = _f64(grid); u = _f64(u)
    dim, nb1 = grid.shape
    x = np.zeros(dim); bins = np.zeros(dim, dtype=np.uint8)
    j = lib().or_vegas_map(_dp(grid), dim, nb1 - 1, _dp(u), _dp(x), bins.ctypes.data_as(_U8))
    return x, bins, j


def vegas_refine(hist: np.ndarray, grid: np.ndarray, alpha: float = 1.5) -> np.ndarray:
    hist = _f64(hist); g = _f64(grid).copy()
    dim, nb1 = g.shape
    lib().or_vegas_refine(_dp(hist), _dp(g), dim, nb1 - 1, alpha)
    return g


def vegas_combine(I, var):
    I = _f64(I); var = _f64(var)
    m, e, c = C.c_double(), C.c_double(), C.c_double()
    lib().or_vegas_combine(len(I), _dp(I), _dp(var), C.byref(m), C.byref(e), C.byref(c))
    return m.value, e.value, c.value


def parton_map(x0: float, v: float, tau0: float):
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    lib().or_parton_map(x0, v, tau0, C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def rambo(n: int, sqrt_shat: float, masses, u):
    m = _f64(masses); u = _f64(u)
    p = np.zeros((n, 4)); w = C.c_double()
    rc = lib().or_rambo(n, sqrt_shat, _dp(m), _dp(u), _dp(p), C.byref(w))
    if rc:
        raise ValueError("rambo: below threshold")
    return p, w.value


def rambo_massless_volume(n: int, shat: float) -> float:
    return lib().or_rambo_massless_volume(n, shat)


def cuts(proc: int, phys, plab) -> int:
    P = params(phys); p = _f64(plab)
    return lib().or_cuts(proc, C.byref(P), _dp(p))


def muf2(proc: int, phys, p) -> float:
    P = params(phys); p = _f64(p)
    return lib().or_muf2(proc, C.byref(P), _dp(p))


def me2(proc: int, phys, p) -> float:
    P = params(phys); p = _f64(p)
    return lib().or_me2(proc, C.byref(P), _dp(p))


def me2_ee_mumu_closed(phys, p) -> float:
    P = params(phys); p = _f64(p)
    return lib().or_me2_ee_mumu_closed(C.byref(P), _dp(p))


def me2_gg_tt_closed(mt, gs, p) -> float:
    return lib().or_me2_gg_tt_closed(mt, gs, _dp(_f64(p)))


def me2_uu_tt_closed(mt, gs, p) -> float:
    return lib().or_me2_uu_tt_closed(mt, gs, _dp(_f64(p)))


def me2_uu_tt_diagram(mt, gs, p) -> float:
    return lib().or_me2_uu_tt_diagram(mt, gs, _dp(_f64(p)))


def me2_ug_ttu(mt, gs, p) -> float:
    return lib().or_me2_ug_ttu(mt, gs, _dp(_f64(p)))


def amp2_ug_ttu_ward(mt, gs, p) -> float:
    return lib().or_amp2_ug_ttu_ward(mt, gs, _dp(_f64(p)))


def me2_bg(k: int, p_all, n_in_gluons: int, m: float, gs: float) -> float:
    return lib().or_me2_bg(k, _dp(_f64(p_all)), n_in_gluons, m, gs)


def bg_partial(kg, eps, p3, p4, m, gs, s3, s4, perm) -> complex:
    kg = _f64(kg); k = kg.shape[0]
    e = np.zeros((k, 4, 2)); eps = np.asarray(eps, dtype=complex)
    e[..., 0] = eps.real; e[..., 1] = eps.imag
    e = _f64(e)
    pr = (C.c_int * k)(*perm)
    out = np.zeros(2)
    lib().or_bg_partial(k, _dp(kg), _dp(e), _dp(_f64(p3)), _dp(_f64(p4)), m, gs, s3, s4, pr, _dp(out))
    return complex(out[0], out[1])


def colour_matrix(k: int) -> np.ndarray:
    n = math.factorial(k)
    Cm = np.zeros((n, n))
    lib().or_colour_matrix(k, _dp(Cm))
    return Cm


def gellmann_T(a: int) -> np.ndarray:
    o = np.zeros(18)
    lib().or_gellmann_T(a, _dp(o))
    return (o[0::2] + 1j * o[1::2]).reshape(3, 3)


def event(proc: int, phys, pdf: Pdf, grid: np.ndarray, ev: int, iteration: int = 0, mask=None) -> OrEvent:
    P = params(phys); g = _f64(grid); o = OrEvent()
    mo = C.c_int(int(mask)) if mask is not None else None
    rc = lib().or_event(proc, C.byref(P), C.byref(pdf.c), _dp(g), ev, iteration,
                        C.byref(mo) if mo is not None else None, C.byref(o))
    if rc:
        raise ValueError("or_event failed")
    return o


def events(proc: int, phys, pdf: Pdf, grid: np.ndarray, idx, iteration: int = 0, n_threads: int = 0):
    """event() for every index in idx, computed in parallel; a list of OrEvent."""
    P = params(phys); g = _f64(grid)
    ev = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    out = (OrEvent * max(len(ev), 1))()
    rc = lib().or_events(proc, C.byref(P), C.byref(pdf.c), _dp(g), ev.ctypes.data_as(C.POINTER(C.c_uint64)),
                         len(ev), iteration, out, n_threads)
    if rc:
        raise ValueError("or_events failed")
    return [out[i] for i in range(len(ev))]


def vegas_pass(proc: int, phys, pdf: Pdf, grid: np.ndarray, n: int, iteration: int = 0,
               mask_in=None, want_mask=False, n_threads: int = 0):
    P = params(phys); g = _f64(grid)
    dim = g.shape[0]; nb = g.shape[1] - 1
    hist = np.zeros((dim, nb))
    sw, sw2 = C.c_double(), C.c_double(); npass = C.c_int64()
    mi = None
    if mask_in is not None:
        mi = np.ascontiguousarray(mask_in, dtype=np.uint8)
    mo = np.zeros(n, dtype=np.uint8) if want_mask else None
    rc = lib().or_pass(proc, C.byref(P), C.byref(pdf.c), _dp(g), n, iteration,
                       mi.ctypes.data_as(_U8) if mi is not None else None,
                       mo.ctypes.data_as(_U8) if mo is not None else None,
                       C.byref(sw), C.byref(sw2), _dp(hist), C.byref(npass), n_threads)
    if rc:
        raise RuntimeError(f"or_pass failed ({rc})")
    return dict(sum_w=sw.value, sum_w2=sw2.value, hist=hist, n_pass=npass.value, mask=mo)


def obs_bin(px: float, py: float, nobs: int, lo: float, hi: float) -> int:
    return lib().or_obs_bin(px, py, nobs, lo, hi)


def vegas_pass_obs(proc: int, phys, pdf: Pdf, grid: np.ndarray, n: int, nobs: int, lo: float, hi: float,
                   iteration: int = 0, n_threads: int = 0):
    """One pass with the observable histogram: obs [nobs + 2][2] (sum w/N, sum (w/N)^2)."""
    P = params(phys); g = _f64(grid)
    sw, sw2 = C.c_double(), C.c_double()
    obs = np.zeros((nobs + 2, 2))
    rc = lib().or_pass_obs(proc, C.byref(P), C.byref(pdf.c), _dp(g), n, iteration, nobs, lo, hi,
                           C.byref(sw), C.byref(sw2), _dp(obs), n_threads)
    if rc:
        raise RuntimeError(f"or_pass_obs failed ({rc})")
    return dict(sum_w=sw.value, sum_w2=sw2.value, obs=obs)


def integrate_obs(proc: int, phys, pdf: Pdf, n: int, n_iter: int, nobs: int, lo: float, hi: float,
                  n_threads: int = 0):
    """VEGAS integration with the observable histogram (combined over iterations)."""
    P = params(phys); res = OrResult()
    h = np.zeros(nobs + 2); e = np.zeros(nobs + 2); it = np.zeros((n_iter, nobs + 2, 2))
    rc = lib().or_integrate_obs(proc, C.byref(P), C.byref(pdf.c), n, n_iter, nobs, lo, hi, _dp(h), _dp(e),
                                _dp(it), C.byref(res), n_threads)
    if rc:
        raise RuntimeError(f"or_integrate_obs failed ({rc})")
    return dict(sigma=res.sigma, error=res.error, chi2dof=res.chi2dof, n_pass=res.n_pass,
                hist=h, err=e, per_iter=it)


def integrate(proc: int, phys, pdf: Pdf, n: int, n_iter: int, n_threads: int = 0):
    P = params(phys); info = proc_info(proc)
    grid = np.zeros((info.dim, phys.n_bins + 1))
    per = np.zeros((n_iter, 2)); res = OrResult()
    rc = lib().or_integrate(proc, C.byref(P), C.byref(pdf.c), n, n_iter, _dp(grid), _dp(per),
                            C.byref(res), n_threads)
    if rc:
        raise RuntimeError(f"or_integrate failed ({rc})")
    return dict(sigma=res.sigma, error=res.error, chi2dof=res.chi2dof, n_pass=res.n_pass,
                grid=grid, per_iter=per)

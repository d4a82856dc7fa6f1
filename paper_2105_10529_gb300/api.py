"""Python front end of the C ABI (argument marshalling only; every step of
the integrand runs in the library's CUDA kernels).  PyTorch provides device
memory and the stream."""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _lib
from ._lib import MfConfig, MfCuts, MfError, MfEventArrays, MfObs, MfResult
from . import inputs as IN


def _torch():
    import torch
    return torch


def _check(ctx_ptr, rc: int):
    if rc != 0:
        msg = _lib.lib().mf_last_error(ctx_ptr)
        raise MfError(rc, msg.decode() if msg else "")


def process_info(process: int):
    n_ext, dim = C.c_int(), C.c_int()
    rc = _lib.lib().mf_process_info(process, C.byref(n_ext), C.byref(dim))
    if rc:
        raise MfError(rc, f"process {process}")
    return n_ext.value, dim.value


def _cuts(cuts):
    """None, an MfCuts, or (pt_min, eta_max, dr_min) -> ctypes pointer or None."""
    if cuts is None:
        return None
    if not isinstance(cuts, MfCuts):
        cuts = MfCuts(*[float(x) for x in cuts])
    return C.byref(cuts)


def _result(r: MfResult) -> dict:
    return dict(sigma=r.sigma_pb, error=r.error_pb, chi2dof=r.chi2_dof, n_events=r.n_events_total,
                n_pass=r.n_pass, n_nan=r.n_nan, dsigma_dmt=r.dsigma_dmt, dsigma_dmt_error=r.dsigma_dmt_error,
                dsigma_dalphas=r.dsigma_dalphas)


def make_config(physics: Optional[IN.Physics] = None, precision: int = _lib.MF_MIXED) -> MfConfig:
    cfg = MfConfig()
    _lib.lib().mf_default_config(C.byref(cfg))
    if physics is not None:
        for k in ("mt", "alpha_s", "mz", "wz", "alpha_em_inv", "gf", "pt_min", "eta_max", "dr_min",
                  "seed", "channel", "n_bins", "alpha"):
            setattr(cfg, k, getattr(physics, k))
    cfg.precision = precision
    return cfg


class Context:
    """Owns an mf_ctx bound to the current CUDA device and torch stream."""

    def __init__(self, physics: Optional[IN.Physics] = None, pdf_grid: Optional[np.ndarray] = None,
                 precision: int = _lib.MF_MIXED, stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("madflow_gb300 needs a CUDA device (no CPU fallback)")
        self.physics = physics or IN.Physics()
        grid = IN.make_pdf_grid() if pdf_grid is None else np.ascontiguousarray(pdf_grid, dtype=np.float64)
        self._grid = grid
        nf, nx, nq = grid.shape
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        self.cfg = make_config(self.physics, precision)
        ptr = C.c_void_p()
        rc = _lib.lib().mf_create(C.byref(ptr), C.byref(self.cfg), grid.ctypes.data_as(C.POINTER(C.c_double)),
                                  nf, nx, nq, IN.PDF_X_MIN, IN.PDF_Q2_MIN, IN.PDF_Q2_MAX,
                                  C.c_void_p(s.cuda_stream))
        if rc:
            raise MfError(rc, "mf_create failed")
        self.ptr = ptr

    def close(self):
        if getattr(self, "ptr", None):
            _lib.lib().mf_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision: int):
        _check(self.ptr, _lib.lib().mf_set_precision(self.ptr, precision))

    def set_schedule(self, sched: int):
        _check(self.ptr, _lib.lib().mf_set_schedule(self.ptr, sched))

    def set_helicity_split(self, parts: int):
        """Threads per event of the heavy integrand (1 or 2), as mf_set_helicity_split."""
        _check(self.ptr, _lib.lib().mf_set_helicity_split(self.ptr, parts))

    def set_helicity_sampling(self, n_samples: int, stream: int = 0):
        """Helicity configurations sampled per event of g g -> t tbar g g g (0: the full sum), and
        the stream of the draws, as mf_set_helicity_sampling."""
        _check(self.ptr, _lib.lib().mf_set_helicity_sampling(self.ptr, int(n_samples), int(stream) & 0xFFFFFFFF))

    def set_observable(self, n_bins: int = 0, lo: float = 0.0, hi: float = 0.0):
        """p_T histogram of the first final-state particle for the next integrate calls
        (n_bins = 0 disables), as mf_set_observable."""
        spec = MfObs(int(n_bins), float(lo), float(hi)) if n_bins else None
        self._obs_n = 0
        _check(self.ptr, _lib.lib().mf_set_observable(self.ptr, C.byref(spec) if spec is not None else None))
        self._obs_n = int(n_bins)

    def observable(self, n_iter: Optional[int] = None):
        """The last integrate call's histogram: (pb per bin [n+2], errors [n+2]) and, with
        n_iter, each iteration's [n_iter][n+2][2] (sum w/N, variance)."""
        n2 = getattr(self, "_obs_n", 0) + 2
        h = np.zeros(n2); e = np.zeros(n2)
        it = np.zeros((n_iter, n2, 2)) if n_iter else None
        dp = C.POINTER(C.c_double)
        _check(self.ptr, _lib.lib().mf_get_observable(self.ptr, h.ctypes.data_as(dp), e.ctypes.data_as(dp),
                                                      it.ctypes.data_as(dp) if it is not None else None))
        return (h, e) if it is None else (h, e, it)

    def device_status(self):
        """Raises MfError(MF_ERR_TIMEOUT) if a bounded device wait ran out since the last check."""
        _check(self.ptr, _lib.lib().mf_device_status(self.ptr))

    def selftest_wait(self, iterations: int = 4096) -> int:
        """Status of the bounded-wait self-test (MF_ERR_TIMEOUT = 3 when the expiry is detected)."""
        return _lib.lib().mf_selftest_wait(self.ptr, iterations)

    def set_pdf(self, grid_host: np.ndarray):
        """Upload a host PDF grid (same shape as at creation); asynchronous on the stream."""
        g = np.ascontiguousarray(grid_host, dtype=np.float64)
        self._pending_pdf = g
        _check(self.ptr, _lib.lib().mf_set_pdf(self.ptr, g.ctypes.data_as(C.POINTER(C.c_double))))

    def integrate(self, process: int, sqrt_s: float, n_events: int, n_iter: int, want_grid: bool = False,
                  want_grads: bool = False, cuts=None):
        """mf_integrate; cuts: None (the configuration's) or (pt_min, eta_max, dr_min)."""
        res = MfResult()
        it = np.zeros((n_iter, 2))
        _, dim = process_info(process)
        grid = np.zeros((dim, self.cfg.n_bins + 1)) if want_grid else None
        rc = _lib.lib().mf_integrate(self.ptr, process, sqrt_s, _cuts(cuts), n_events, n_iter, int(want_grads),
                                     C.byref(res), it.ctypes.data_as(C.POINTER(C.c_double)),
                                     grid.ctypes.data_as(C.POINTER(C.c_double)) if grid is not None else None)
        out = _result(res)
        out.update(per_iter=it, grid=grid, status=rc)
        _check(self.ptr, rc)
        return out

    def integrate_grid(self, process: int, sqrt_s: float, n_events: int, n_iter: int, grid, first_iteration: int = 0,
                       want_grads: bool = False, cuts=None):
        """mf_integrate_grid: iterations from a host grid [dim][n_bins+1], Philox iterations from
        first_iteration on; returns the integrate() dict with the final grid."""
        res = MfResult()
        it = np.zeros((n_iter, 2))
        g_in = np.ascontiguousarray(grid, dtype=np.float64)
        g_out = np.zeros_like(g_in)
        dp = C.POINTER(C.c_double)
        rc = _lib.lib().mf_integrate_grid(self.ptr, process, sqrt_s, _cuts(cuts), n_events, n_iter, first_iteration,
                                          g_in.ctypes.data_as(dp), int(want_grads), C.byref(res),
                                          it.ctypes.data_as(dp), g_out.ctypes.data_as(dp))
        out = _result(res)
        out.update(per_iter=it, grid=g_out, status=rc)
        _check(self.ptr, rc)
        return out

    def integrate_batch(self, processes, n_events, sqrt_s: float, n_iter: int, want_grids: bool = False,
                        want_grads: bool = False, cuts=None):
        """Several channels in one persistent launch per iteration (mf_integrate_batch).
        Returns (total dict, list of per-channel dicts)."""
        n_ch = len(processes)
        procs = (C.c_int * n_ch)(*[int(p) for p in processes])
        ns = (C.c_longlong * n_ch)(*[int(n) for n in n_events])
        per = (MfResult * n_ch)()
        tot = MfResult()
        grids = np.zeros((n_ch, 18, self.cfg.n_bins + 1)) if want_grids else None
        rc = _lib.lib().mf_integrate_batch(self.ptr, n_ch, procs, ns, sqrt_s, _cuts(cuts), n_iter, int(want_grads),
                                           per, C.byref(tot),
                                           grids.ctypes.data_as(C.POINTER(C.c_double)) if grids is not None else None)
        _check(self.ptr, rc)
        d = _result
        chans = [d(per[i]) for i in range(n_ch)]
        if grids is not None:
            for i, p in enumerate(processes):
                chans[i]["grid"] = grids[i, :process_info(p)[1]].copy()
        return d(tot), chans

    def batch_pass(self, processes, n_events, sqrt_s: float, grids, iteration: int = 0, want_events: bool = False,
                   fields=None):
        """One pass of a batch at caller grids (mf_batch_pass): grids [n_ch][18][n_bins+1] (device
        tensor; each channel's first dim rows used).  Returns (sums [n_ch][2 + 18 n_bins], list of
        per-channel event dicts or None)."""
        torch = _torch()
        n_ch = len(processes)
        dev = torch.device("cuda", torch.cuda.current_device())
        nb = self.cfg.n_bins
        grids = grids.to(device=dev, dtype=torch.float64).contiguous()
        assert tuple(grids.shape) == (n_ch, 18, nb + 1)
        sums = torch.zeros((n_ch, 2 + 18 * nb), dtype=torch.float64, device=dev)
        procs = (C.c_int * n_ch)(*[int(p) for p in processes])
        ns = (C.c_longlong * n_ch)(*[int(n) for n in n_events])
        evs, arr = None, None
        if want_events:
            fields = fields or ("u", "x", "bins", "w", "mask", "me2", "momenta")
            evs, arr = [], (MfEventArrays * n_ch)()
            for i, p in enumerate(processes):
                n_ext, dim = process_info(p)
                n = int(n_events[i])
                shapes = dict(u=((n, dim), torch.float64), x=((n, dim), torch.float64),
                              bins=((n, dim), torch.uint8), w=((n,), torch.float64), mask=((n,), torch.uint8),
                              me2=((n,), torch.float64), momenta=((n, n_ext, 4), torch.float64))
                e = {f: torch.empty(*shapes[f][0], dtype=shapes[f][1], device=dev) for f in fields}
                evs.append(e)
                arr[i] = MfEventArrays(**{f: C.c_void_p(e[f].data_ptr()) if f in e else None
                                          for f, _ in MfEventArrays._fields_})
        rc = _lib.lib().mf_batch_pass(self.ptr, n_ch, procs, ns, sqrt_s, C.c_void_p(grids.data_ptr()), iteration,
                                      C.c_void_p(sums.data_ptr()), arr)
        _check(self.ptr, rc)
        return sums, evs

    def batch_grad(self, processes, n_events, sqrt_s: float, iteration: int, cuts=None):
        """Derivative passes at the grids of the last integrate_batch: array [n_ch + 1, 4] of
        (sigma_hat, d sigma_hat/d m_t, its MC error, d sigma_hat/d alpha_s); last row = sum."""
        n_ch = len(processes)
        procs = (C.c_int * n_ch)(*[int(p) for p in processes])
        ns = (C.c_longlong * n_ch)(*[int(n) for n in n_events])
        out = np.zeros((n_ch + 1, 4))
        _check(self.ptr, _lib.lib().mf_batch_grad(self.ptr, n_ch, procs, ns, sqrt_s, _cuts(cuts), iteration,
                                                  out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def set_batch_schedule(self, mode: int, sched: int, tile_heavy: int, tile_light: int, ctas_per_sm: int = 0,
                           hsplit: int = 1):
        _check(self.ptr, _lib.lib().mf_set_batch_schedule(self.ptr, mode, sched, tile_heavy, tile_light,
                                                           ctas_per_sm, hsplit))

    def autotune_batch(self, processes, n_events, sqrt_s: float):
        """Pick the batch schedule by timing: (mode, sched, tile_heavy, tile_light, ctas_per_sm, hsplit)."""
        n_ch = len(processes)
        procs = (C.c_int * n_ch)(*[int(p) for p in processes])
        ns = (C.c_longlong * n_ch)(*[int(n) for n in n_events])
        ch = (C.c_int * 6)()
        _check(self.ptr, _lib.lib().mf_autotune_batch(self.ptr, n_ch, procs, ns, sqrt_s, ch))
        return tuple(ch)

    def vegas_pass(self, process: int, sqrt_s: float, grid, n_events: int, ev_offset: int = 0,
                   iteration: int = 0, mask_in=None, want_events: bool = False, fields=None):
        """One pass at a device grid; returns (sums tensor, events dict or None)."""
        torch = _torch()
        n_ext, dim = process_info(process)
        dev = torch.device("cuda", torch.cuda.current_device())
        grid = grid.to(device=dev, dtype=torch.float64).contiguous()
        sums = torch.empty(2 + dim * self.cfg.n_bins, dtype=torch.float64, device=dev)
        ev = None
        evs = None
        if want_events:
            fields = fields or ("u", "x", "bins", "w", "mask", "me2", "momenta")
            shapes = dict(u=((n_events, dim), torch.float64), x=((n_events, dim), torch.float64),
                          bins=((n_events, dim), torch.uint8), w=((n_events,), torch.float64),
                          mask=((n_events,), torch.uint8), me2=((n_events,), torch.float64),
                          momenta=((n_events, n_ext, 4), torch.float64))
            evs = {f: torch.empty(*shapes[f][0], dtype=shapes[f][1], device=dev) for f in fields}
            ev = MfEventArrays(**{f: C.c_void_p(evs[f].data_ptr()) if f in evs else None
                                  for f, _ in MfEventArrays._fields_})
        mptr = None
        if mask_in is not None:
            mask_in = mask_in.to(device=dev, dtype=torch.uint8).contiguous()
            mptr = C.c_void_p(mask_in.data_ptr())
        rc = _lib.lib().mf_vegas_pass(self.ptr, process, sqrt_s, C.c_void_p(grid.data_ptr()), n_events, ev_offset,
                                      iteration, mptr, C.c_void_p(sums.data_ptr()),
                                      C.byref(ev) if ev is not None else None)
        _check(self.ptr, rc)
        return sums, evs

    def set_couplings(self, mt: float, alpha_s: float):
        _check(self.ptr, _lib.lib().mf_set_couplings(self.ptr, float(mt), float(alpha_s)))
        self.cfg.mt, self.cfg.alpha_s = float(mt), float(alpha_s)

    def vegas_pass_grad(self, process: int, sqrt_s: float, grid, n_events: int, ev_offset: int = 0,
                        iteration: int = 0, mask_in=None):
        """Derivative pass at a fixed grid and base-point masks: tensor [4] =
        (sigma_hat, d sigma_hat/d m_t, sum (dw/dm_t / N)^2, d sigma_hat/d alpha_s)."""
        torch = _torch()
        dev = torch.device("cuda", torch.cuda.current_device())
        grid = grid.to(device=dev, dtype=torch.float64).contiguous()
        out = torch.empty(4, dtype=torch.float64, device=dev)
        mptr = None
        if mask_in is not None:
            mask_in = mask_in.to(device=dev, dtype=torch.uint8).contiguous()
            mptr = C.c_void_p(mask_in.data_ptr())
        rc = _lib.lib().mf_vegas_pass_grad(self.ptr, process, sqrt_s, C.c_void_p(grid.data_ptr()), n_events,
                                           ev_offset, iteration, mptr, C.c_void_p(out.data_ptr()))
        _check(self.ptr, rc)
        return out

    def evaluate_grad(self, process: int, momenta):
        """(|M|^2 [n], d|M|^2/dp [n, n_ext, 4]) of momenta [n, n_ext, 4] on the device."""
        torch = _torch()
        mom = momenta.to(dtype=torch.float64).contiguous()
        n = mom.shape[0]
        me = torch.empty(n, dtype=torch.float64, device=mom.device)
        dme = torch.empty_like(mom)
        rc = _lib.lib().mf_evaluate(self.ptr, process, C.c_void_p(mom.data_ptr()), n, C.c_void_p(me.data_ptr()),
                                    C.c_void_p(dme.data_ptr()))
        _check(self.ptr, rc)
        return me, dme

    def helicity_profile(self, process: int, momenta):
        """Per-helicity averaged |M_h|^2 [n, 2^n_ext] of momenta [n, n_ext, 4] (mf_helicity_profile)."""
        torch = _torch()
        mom = momenta.to(dtype=torch.float64).contiguous()
        n, n_ext = mom.shape[0], mom.shape[1]
        out = torch.empty((n, 1 << n_ext), dtype=torch.float64, device=mom.device)
        rc = _lib.lib().mf_helicity_profile(self.ptr, process, C.c_void_p(mom.data_ptr()), n, C.c_void_p(out.data_ptr()))
        _check(self.ptr, rc)
        return out

    def evaluate(self, process: int, momenta):
        """Averaged |M|^2 of momenta [n, n_ext, 4] (float64, on the device)."""
        torch = _torch()
        mom = momenta.to(dtype=torch.float64).contiguous()
        n = mom.shape[0]
        out = torch.empty(n, dtype=torch.float64, device=mom.device)
        rc = _lib.lib().mf_evaluate(self.ptr, process, C.c_void_p(mom.data_ptr()), n, C.c_void_p(out.data_ptr()), None)
        _check(self.ptr, rc)
        return out


def measure_fma_peak(precision: int, stream=None) -> float:
    """FMA throughput of the current device in TFLOP/s (mf_measure_fma_peak):
    FP32 for MF_MIXED, FP64 for MF_FP64."""
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double(0.0)
    rc = _lib.lib().mf_measure_fma_peak(int(precision), C.c_void_p(s.cuda_stream), C.byref(out))
    if rc:
        raise MfError(rc, "mf_measure_fma_peak failed")
    return float(out.value)


DF_FUNCTIONS = {"exp": 0, "log": 1, "sqrt": 2, "sinpi": 3, "cospi": 4, "recip": 5, "square": 6}


def selftest_df(fn: str, x):
    """The double-float function fn (a key of DF_FUNCTIONS) of the mixed-precision kinematics
    at the points x (a float64 CUDA tensor), as doubles (mf_selftest_df)."""
    torch = _torch()
    if x.dtype != torch.float64 or not x.is_cuda:
        raise ValueError("x: a float64 CUDA tensor")
    x = x.contiguous()
    y = torch.empty_like(x)
    s = torch.cuda.current_stream()
    rc = _lib.lib().mf_selftest_df(DF_FUNCTIONS[fn], C.c_void_p(x.data_ptr()), x.numel(), C.c_void_p(y.data_ptr()),
                                   C.c_void_p(s.cuda_stream))
    if rc:
        raise MfError(rc, "mf_selftest_df failed")
    return y


def integrate(process: int, sqrt_s: float, n_events: int, n_iter: int, physics: Optional[IN.Physics] = None,
              precision: int = _lib.MF_MIXED):
    """One-shot integrate(process, sqrt_s, n_events, n_iter) -> sigma, error (Sec. 2.1)."""
    ctx = Context(physics, precision=precision)
    try:
        return ctx.integrate(process, sqrt_s, n_events, n_iter)
    finally:
        ctx.close()

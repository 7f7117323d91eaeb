"""GB300-native log-likelihood of Gaussian processes with integrated, possibly
overlapping exposures (Rubenzahl, Hattori et al., arXiv 2601.02527).

This package is a thin binding over ``libgpss.so`` (CUDA, sm_103a; C ABI in
``include/gpss.h``): arguments are marshalled here and every step of the
computation runs in the library's kernels.  PyTorch supplies device memory and
streams.  There is no CPU fallback: if the library is missing or no CUDA
device is present, calls raise.

``Model`` holds one event stream (exposure averages, or instantaneous
measurements with t_end == t_start) and offers the log-likelihood, its
gradient with respect to the hyperparameters and the exposure windows, the
conditioned value of every measurement, predictions at arbitrary times and an
autotuner; ``loglik`` wraps the gradient in a ``torch.autograd.Function``.
Kernel terms: SHO (any Q > 0), Matern-3/2, and a product of two SHOs.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpss.so")

SHO = 1
MATERN32 = 2
SHO_PRODUCT = 3

STATUS = {0: "ok", 1: "invalid argument", 2: "series offsets not sorted",
          3: "an instrument's exposures overlap each other",
          4: "unsupported model shape or parameter regime", 5: "out of memory",
          6: "CUDA runtime error", 7: "non-positive or non-finite innovation variance",
          8: "bounded device wait timed out",
          9: "problem needs more than the fixed scratch of gp_ss_loglik_noalloc"}

# every function declared in include/gpss.h
EXPORTS = ["gp_ss_build_model", "gp_ss_loglik", "gp_ss_loglik_grad", "gp_ss_loglik_batched",
           "gp_ss_loglik_grad_batched", "gp_ss_loglik_grad_host", "gp_ss_model_info",
           "gp_ss_set_chunk_len", "gp_ss_last_error_series", "gp_ss_free_model",
           "gp_ss_status_string", "gp_ss_discretize", "gp_ss_set_timing", "gp_ss_get_timing",
           "gp_ss_loglik_noalloc", "gp_ss_launch_count", "gp_ss_autotune", "gp_ss_condition",
           "gp_ss_predict", "gp_ss_measure_fp32_peak", "gp_ss_span_element",
           "gp_ss_span_loglik", "gp_ss_build_events"]

PHASES = ["elem", "scan", "grad", "convert", "plain"]


class GPSSError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)} (status {code})")


class _KernelSpec(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_int), ("terms", ctypes.POINTER(ctypes.c_int)),
                ("integral_layout", ctypes.c_int)]


class _Tuning(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int), ("chunk_len", ctypes.c_int),
                ("chunk_combine", ctypes.c_int), ("ckpt_interval", ctypes.c_int),
                ("threads_per_series", ctypes.c_int), ("n_tried", ctypes.c_int),
                ("ms", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("schedule", ctypes.c_int),
                ("threads_per_series", ctypes.c_int), ("chunk_len", ctypes.c_int),
                ("ckpt_interval", ctypes.c_int), ("debug_checks", ctypes.c_int),
                ("chunk_combine", ctypes.c_int), ("step_cache", ctypes.c_int),
                ("combine_precision", ctypes.c_int)]


_lib = None


def load_library(path: str | None = None):
    """Load libgpss.so (built by ``paper_2601_02527_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libgpss.so not found at {p}; build it with "
                           "`python -m paper_2601_02527_gb300.build`")
    lib = ctypes.CDLL(p)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    P = ctypes.POINTER
    lib.gp_ss_build_model.argtypes = [P(_KernelSpec), i32, vp, vp, vp, vp, vp, vp, P(_Options),
                                      P(vp)]
    lib.gp_ss_loglik.argtypes = [vp, vp, i32, i32, vp, vp]
    lib.gp_ss_loglik_grad.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp]
    lib.gp_ss_loglik_batched.argtypes = [vp, vp, i32, i32, vp, vp]
    lib.gp_ss_loglik_grad_batched.argtypes = [vp, vp, i32, i32, vp, vp, vp]
    lib.gp_ss_loglik_grad_host.argtypes = [vp, vp, i32, i32, vp, vp, i32, vp]
    lib.gp_ss_model_info.argtypes = [vp, P(i32), P(i64), P(i64), P(i32), P(i32), P(i32), P(i32)]
    lib.gp_ss_set_chunk_len.argtypes = [vp, i32]
    lib.gp_ss_last_error_series.argtypes = [vp, P(i64), P(i32)]
    lib.gp_ss_free_model.argtypes = [vp]
    lib.gp_ss_free_model.restype = None
    lib.gp_ss_launch_count.argtypes = [P(i64)]
    lib.gp_ss_condition.argtypes = [vp, vp, i32, i32, vp, vp, vp]
    lib.gp_ss_predict.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp]
    lib.gp_ss_autotune.argtypes = [vp, vp, i32, i32, i32, i32, P(_Tuning), vp]
    lib.gp_ss_status_string.argtypes = [i32]
    lib.gp_ss_status_string.restype = ctypes.c_char_p
    lib.gp_ss_discretize.argtypes = [P(_KernelSpec), i32, vp, vp, i32, vp, vp, vp]
    lib.gp_ss_set_timing.argtypes = [vp, i32]
    lib.gp_ss_loglik_noalloc.argtypes = [vp, vp, i32, i32, vp, vp]
    lib.gp_ss_get_timing.argtypes = [vp, vp, vp]
    lib.gp_ss_measure_fp32_peak.argtypes = [P(ctypes.c_double), P(i32), vp]
    lib.gp_ss_span_element.argtypes = [vp, vp, i32, i32, i32, i32, vp, vp]
    lib.gp_ss_span_loglik.argtypes = [vp, vp, i32, i32, vp, vp]
    lib.gp_ss_build_events.argtypes = [i64, vp, vp, vp, vp, vp, P(i64), vp, vp, vp, P(i32)]
    _lib = lib
    return lib


def _check(code, what):
    if code != 0:
        raise GPSSError(code, what)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _spec(terms, layout):
    arr = (ctypes.c_int * len(terms))(*[int(t) for t in terms])
    return _KernelSpec(len(terms), arr, int(layout)), arr


def n_params_for(terms) -> int:
    return sum({SHO: 3, SHO_PRODUCT: 5}.get(int(t), 2) for t in terms) + 1


class Model:
    """An event-stream model on the current CUDA device (gp_ss_build_model).

    ``offsets`` (int64, n_series+1) delimits the series in the concatenated
    per-measurement arrays ``t_start``, ``t_end`` (float64), ``y``, ``yerr``
    (float32) and optional ``instrument`` (int32 slot labels).
    """

    def __init__(self, terms, offsets, t_start, t_end, y, yerr, instrument=None, layout=0,
                 precision=32, schedule=0, chunk_len=0, combine=0, ckpt_interval=0,
                 step_cache=0, combine_precision=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        lib = load_library()
        self.terms = [int(t) for t in terms]
        self.layout = int(layout)
        self.n_params = n_params_for(self.terms)
        offs = np.ascontiguousarray(offsets, np.int64)
        self.offsets = offs.copy()
        self._meas_series = None
        ts = np.ascontiguousarray(t_start, np.float64)
        te = np.ascontiguousarray(t_end, np.float64)
        yy = np.ascontiguousarray(y, np.float32)
        ye = np.ascontiguousarray(yerr, np.float32)
        inst = None if instrument is None else np.ascontiguousarray(instrument, np.int32)
        spec, self._spec_arr = _spec(self.terms, self.layout)
        opts = _Options(int(precision), int(schedule), 0, int(chunk_len), int(ckpt_interval), 0,
                        int(combine), int(step_cache), int(combine_precision))
        h = ctypes.c_void_p()
        self.device = torch.cuda.current_device()
        rc = lib.gp_ss_build_model(ctypes.byref(spec), len(offs) - 1, offs.ctypes.data,
                                   ts.ctypes.data, te.ctypes.data, yy.ctypes.data,
                                   ye.ctypes.data, None if inst is None else inst.ctypes.data,
                                   ctypes.byref(opts), ctypes.byref(h))
        _check(rc, "gp_ss_build_model")
        self._h = h
        self._lib = lib
        self.info = self._info()

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(wl.terms, wl.offsets, wl.t_start, wl.t_end, wl.y, wl.yerr, wl.instrument,
                   layout=wl.layout, **kw)

    def _info(self):
        ns, nd, np_, sd, sl, nc = (ctypes.c_int() for _ in range(6))
        nm, ne = ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.gp_ss_model_info(self._h, ctypes.byref(ns), ctypes.byref(nm),
                                          ctypes.byref(ne), ctypes.byref(np_), ctypes.byref(sd),
                                          ctypes.byref(sl), ctypes.byref(nc)), "gp_ss_model_info")
        return dict(n_series=ns.value, n_meas=nm.value, n_events=ne.value,
                    n_params=np_.value, state_dim=sd.value, n_slots=sl.value,
                    n_chunks=nc.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gp_ss_free_model(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_out(self, theta, per_series):
        n_sets = theta.shape[0]
        return self.info["n_series"] if per_series else n_sets * self.info["n_series"]

    def _theta(self, theta):
        import torch
        if not (isinstance(theta, torch.Tensor) and theta.is_cuda):
            raise TypeError("theta must be a CUDA tensor")
        if theta.device.index != self.device:
            raise ValueError(f"theta is on cuda:{theta.device.index}, the model on "
                             f"cuda:{self.device}")
        th = theta.detach().to(torch.float32).contiguous()
        if th.dim() != 2 or th.shape[1] != self.n_params:
            raise ValueError(f"theta must be [n_sets, {self.n_params}]")
        return th

    def _check_out(self, t, what, dtype, numel):
        """A caller-supplied output buffer must be a contiguous tensor of the
        given dtype on the model's device with at least ``numel`` elements:
        the kernels write that many values through its pointer."""
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{what} must be a CUDA tensor")
        if t.device.index != self.device:
            raise ValueError(f"{what} is on cuda:{t.device.index}, the model on "
                             f"cuda:{self.device}")
        if t.dtype != dtype:
            raise ValueError(f"{what} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
        if t.numel() < numel:
            raise ValueError(f"{what} holds {t.numel()} elements, {numel} needed")
        return t

    def loglik(self, theta, per_series=True, out=None, stream=None, batched=False):
        """Log-likelihood per output row (float64 CUDA tensor)."""
        import torch
        th = self._theta(theta)
        n = self.n_out(th, per_series)
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=th.device)
        self._check_out(out, "out", torch.float64, n)
        f = self._lib.gp_ss_loglik_batched if batched else self._lib.gp_ss_loglik
        _check(f(self._h, th.data_ptr(), th.shape[0], int(bool(per_series)), out.data_ptr(),
                 _stream_ptr(stream)), "gp_ss_loglik")
        return out

    def measurement_series(self, device):
        """Series index of every measurement (int64 tensor [N] on ``device``)."""
        import torch
        if self._meas_series is None or self._meas_series.device != torch.device(device):
            counts = torch.as_tensor(np.diff(self.offsets), device=device)
            self._meas_series = torch.repeat_interleave(
                torch.arange(len(counts), device=device), counts)
        return self._meas_series

    def loglik_noalloc(self, theta, per_series=True, out=None, stream=None):
        """Log-likelihood through gp_ss_loglik_noalloc: the library allocates
        nothing (its scratch is a fixed 16 MiB array per GPU).  For callers
        that cannot allocate device memory at call time; calls that overlap on
        the GPU share that array and must be serialised."""
        import torch
        th = self._theta(theta)
        n = self.n_out(th, per_series)
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=th.device)
        self._check_out(out, "out", torch.float64, n)
        _check(self._lib.gp_ss_loglik_noalloc(self._h, th.data_ptr(), th.shape[0],
                                              int(bool(per_series)), out.data_ptr(),
                                              _stream_ptr(stream)), "gp_ss_loglik_noalloc")
        return out

    def loglik_grad(self, theta, per_series=True, out=None, grad=None, stream=None,
                    batched=False, exposure=False, dexp=None):
        """(log-likelihood [n_out] float64, gradient [n_out, n_params] float32),
        plus, with ``exposure``, the exposure-window gradient [rows, N, 2] float32
        ((d/d t_start, d/d t_end) per measurement; rows = 1 per series mode, else
        the number of theta sets)."""
        import torch
        th = self._theta(theta)
        n = self.n_out(th, per_series)
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=th.device)
        if grad is None:
            grad = torch.empty(n, self.n_params, dtype=torch.float32, device=th.device)
        if exposure and batched:
            raise ValueError("the exposure gradient is computed by the direct call only")
        self._check_out(out, "out", torch.float64, n)
        self._check_out(grad, "grad", torch.float32, n * self.n_params)
        if exposure:
            rows = 1 if per_series else th.shape[0]
            if dexp is None:
                dexp = torch.empty(rows, self.info["n_meas"], 2, dtype=torch.float32,
                                   device=th.device)
            self._check_out(dexp, "dexp", torch.float32, rows * self.info["n_meas"] * 2)
        if batched:
            rc = self._lib.gp_ss_loglik_grad_batched(self._h, th.data_ptr(), th.shape[0],
                                                     int(bool(per_series)), out.data_ptr(),
                                                     grad.data_ptr(), _stream_ptr(stream))
        else:
            rc = self._lib.gp_ss_loglik_grad(self._h, th.data_ptr(), th.shape[0],
                                             int(bool(per_series)), out.data_ptr(),
                                             grad.data_ptr(),
                                             dexp.data_ptr() if exposure else None,
                                             _stream_ptr(stream))
        _check(rc, "gp_ss_loglik_grad")
        return (out, grad, dexp) if exposure else (out, grad)

    def condition(self, theta, per_series=True, stream=None):
        """(log-likelihood [n_out] float64, conditioned [rows, N, 2] float32):
        the mean and variance of every measurement's exposure average given
        all of its series' data (integrated RTS smoother)."""
        import torch
        th = self._theta(theta)
        out = torch.empty(self.n_out(th, per_series), dtype=torch.float64, device=th.device)
        rows = 1 if per_series else th.shape[0]
        cond = torch.empty(rows, self.info["n_meas"], 2, dtype=torch.float32, device=th.device)
        _check(self._lib.gp_ss_condition(self._h, th.data_ptr(), th.shape[0], int(bool(per_series)),
                                         out.data_ptr(), cond.data_ptr(), _stream_ptr(stream)),
               "gp_ss_condition")
        return out, cond

    def predict(self, theta, t_star, star_offsets, per_series=True, stream=None):
        """(log-likelihood [n_out] float64, prediction [rows, M, 2] float32): mean
        and variance of the latent f(t*) at the test times (series i's at
        t_star[star_offsets[i]:star_offsets[i+1]]) given all the data."""
        import torch
        th = self._theta(theta)
        ts = np.ascontiguousarray(t_star, np.float64)
        so = np.ascontiguousarray(star_offsets, np.int64)
        out = torch.empty(self.n_out(th, per_series), dtype=torch.float64, device=th.device)
        rows = 1 if per_series else th.shape[0]
        pred = torch.empty(rows, len(ts), 2, dtype=torch.float32, device=th.device)
        _check(self._lib.gp_ss_predict(self._h, th.data_ptr(), th.shape[0], int(bool(per_series)),
                                       ts.ctypes.data, so.ctypes.data, out.data_ptr(),
                                       pred.data_ptr(), _stream_ptr(stream)), "gp_ss_predict")
        return out, pred

    def loglik_grad_host(self, theta, per_series=True, reupload_events=False, stream=None):
        """Host-buffer variant: numpy in, numpy out (synchronous)."""
        th = np.ascontiguousarray(theta, np.float32)
        n = self.info["n_series"] if per_series else th.shape[0] * self.info["n_series"]
        ll = np.empty(n, np.float64)
        g = np.empty((n, self.n_params), np.float32)
        _check(self._lib.gp_ss_loglik_grad_host(self._h, th.ctypes.data, th.shape[0],
                                                int(bool(per_series)), ll.ctypes.data,
                                                g.ctypes.data, int(bool(reupload_events)),
                                                _stream_ptr(stream)), "gp_ss_loglik_grad_host")
        return ll, g

    def autotune(self, theta, per_series=True, grad=True, reps=3, stream=None):
        """Time the candidate schedules on this model (gp_ss_autotune), keep the
        fastest and return it as a dict."""
        th = self._theta(theta)
        t = _Tuning()
        _check(self._lib.gp_ss_autotune(self._h, th.data_ptr(), th.shape[0], int(bool(per_series)),
                                        int(bool(grad)), int(reps), ctypes.byref(t),
                                        _stream_ptr(stream)), "gp_ss_autotune")
        self.info = self._info()
        return {f: getattr(t, f) for f, _ in _Tuning._fields_}

    def span_element(self, theta, c_begin, c_end, per_series=True, stream=None):
        """Element of chunks [c_begin, c_end) of this one-series model
        (gp_ss_span_element): float64 CUDA tensor [rows, 2d^2 + 3d + 1]."""
        import torch
        th = self._theta(theta)
        rows = 1 if per_series else th.shape[0]
        d = self.info["state_dim"]
        out = torch.empty(rows, 2 * d * d + 3 * d + 1, dtype=torch.float64, device=th.device)
        _check(self._lib.gp_ss_span_element(self._h, th.data_ptr(), th.shape[0],
                                            int(bool(per_series)), int(c_begin), int(c_end),
                                            out.data_ptr(), _stream_ptr(stream)),
               "gp_ss_span_element")
        return out

    def span_loglik(self, span_elems, stream=None):
        """Log-likelihood per row from the elements of consecutive chunk ranges
        covering the series ([n_spans, rows, NC] float64 CUDA tensor)."""
        import torch
        e = span_elems.contiguous()
        d = self.info["state_dim"]
        if e.dim() != 3 or e.shape[2] != 2 * d * d + 3 * d + 1:
            raise ValueError("span elements must be [n_spans, rows, 2d^2 + 3d + 1]")
        self._check_out(e, "span_elems", torch.float64, e.numel())
        out = torch.empty(e.shape[1], dtype=torch.float64, device=e.device)
        _check(self._lib.gp_ss_span_loglik(self._h, e.data_ptr(), e.shape[0], e.shape[1],
                                           out.data_ptr(), _stream_ptr(stream)),
               "gp_ss_span_loglik")
        return out

    def set_chunk_len(self, chunk_len: int):
        _check(self._lib.gp_ss_set_chunk_len(self._h, int(chunk_len)), "gp_ss_set_chunk_len")
        self.info = self._info()

    def set_timing(self, enable: bool):
        _check(self._lib.gp_ss_set_timing(self._h, int(bool(enable))), "gp_ss_set_timing")

    def get_timing(self):
        """{phase: (total ms, launches)} since the last read (see gp_ss_get_timing)."""
        ms = np.zeros(5, np.float64)
        n = np.zeros(5, np.int64)
        _check(self._lib.gp_ss_get_timing(self._h, ms.ctypes.data, n.ctypes.data),
               "gp_ss_get_timing")
        return {p: (float(ms[i]), int(n[i])) for i, p in enumerate(PHASES)}

    def last_error(self):
        """(first failing output row or -1, status code) of the last call."""
        row, code = ctypes.c_int64(), ctypes.c_int32()
        _check(self._lib.gp_ss_last_error_series(self._h, ctypes.byref(row), ctypes.byref(code)),
               "gp_ss_last_error_series")
        return row.value, code.value


def launch_count() -> int:
    """Kernels the library has launched in this process (host-side count;
    graph replays excluded)."""
    lib = load_library()
    out = ctypes.c_int64()
    _check(lib.gp_ss_launch_count(ctypes.byref(out)), "gp_ss_launch_count")
    return int(out.value)


def measure_fp32_peak(stream=None):
    """(FP32 FMA TFLOP/s measured on the current device, its SM count)."""
    lib = load_library()
    tf, n = ctypes.c_double(), ctypes.c_int()
    _check(lib.gp_ss_measure_fp32_peak(ctypes.byref(tf), ctypes.byref(n), _stream_ptr(stream)),
           "gp_ss_measure_fp32_peak")
    return float(tf.value), int(n.value)


def build_events(t_start, t_end, y, yerr, instrument=None):
    """Host-only event build of one series (gp_ss_build_events): (dt float64,
    tag uint8, meas float64 [n, 3] in event order, n_slots)."""
    lib = load_library()
    ts = np.ascontiguousarray(t_start, np.float64)
    te = np.ascontiguousarray(t_end, np.float64)
    yy = np.ascontiguousarray(y, np.float32)
    ye = np.ascontiguousarray(yerr, np.float32)
    inst = None if instrument is None else np.ascontiguousarray(instrument, np.int32)
    n = len(ts)
    dt = np.empty(max(2 * n, 1), np.float64)
    tag = np.empty(max(2 * n, 1), np.uint8)
    meas = np.empty((max(n, 1), 3), np.float64)
    ne, ns = ctypes.c_int64(), ctypes.c_int()
    _check(lib.gp_ss_build_events(n, ts.ctypes.data, te.ctypes.data, yy.ctypes.data,
                                  ye.ctypes.data, None if inst is None else inst.ctypes.data,
                                  ctypes.byref(ne), dt.ctypes.data, tag.ctypes.data,
                                  meas.ctypes.data, ctypes.byref(ns)), "gp_ss_build_events")
    return dt[:ne.value], tag[:ne.value], meas[:n], ns.value


def discretize(terms, layout, n_slots, theta_row, dt, stream=None):
    """Phi~(dt_k), Q~(dt_k) from the library's per-step discretisation kernel
    (float32, [n, d, d] each) for a CUDA tensor ``dt`` and one parameter row."""
    import torch
    lib = load_library()
    th = theta_row.to(torch.float32).contiguous()
    dtt = dt.to(torch.float32).contiguous()
    spec, _keep = _spec(terms, layout)
    nz = 1 if (layout == 0 or len(terms) == 1) else len(terms)
    d = 2 * len(terms) + n_slots * nz
    phi = torch.empty(dtt.numel(), d, d, dtype=torch.float32, device=dtt.device)
    q = torch.empty_like(phi)
    _check(lib.gp_ss_discretize(ctypes.byref(spec), int(n_slots), th.data_ptr(), dtt.data_ptr(),
                                dtt.numel(), phi.data_ptr(), q.data_ptr(), _stream_ptr(stream)),
           "gp_ss_discretize")
    return phi, q


def _autograd_function():
    import torch

    class LogLikFunction(torch.autograd.Function):
        """Log-likelihood rows with the adjoint gradient as backward, for the
        hyperparameters and (when ``windows`` needs a gradient) the exposure
        windows."""

        @staticmethod
        def forward(ctx, theta, windows, model, per_series):
            want_exp = windows is not None and ctx.needs_input_grad[1]
            if want_exp:
                ll, g, dexp = model.loglik_grad(theta, per_series=per_series, exposure=True)
            else:
                ll, g = model.loglik_grad(theta, per_series=per_series)
                dexp = g.new_empty(0)
            ctx.save_for_backward(g, dexp)
            ctx.want_exp = want_exp
            ctx.model = model
            ctx.per_series = per_series
            ctx.n_sets = theta.shape[0]
            ctx.n_series = model.info["n_series"]
            ctx.wdtype = windows.dtype if windows is not None else None
            return ll

        @staticmethod
        def backward(ctx, gout):
            g, dexp = ctx.saved_tensors
            w = gout.to(torch.float32)[:, None] * g
            if not ctx.per_series:
                w = w.view(ctx.n_sets, ctx.n_series, -1).sum(1)
            gw = None
            if ctx.want_exp:
                sidx = ctx.model.measurement_series(gout.device)
                go = gout.to(torch.float32)
                if ctx.per_series:
                    gw = go[sidx][:, None] * dexp[0]
                else:
                    coef = go.view(ctx.n_sets, ctx.n_series)[:, sidx]
                    gw = (coef[:, :, None] * dexp).sum(0)
                gw = gw.to(ctx.wdtype)
            return w, gw, None, None

    return LogLikFunction


_LLF = None


def loglik(model: Model, theta, per_series=True, windows=None):
    """Differentiable log-likelihood (torch.autograd): rows as ``Model.loglik``.

    ``windows``: optional CUDA tensor [N, 2] of the model's exposure windows
    (t_start, t_end) in measurement order -- the values the model was built
    from; when it requires grad, backward also returns d/d windows."""
    global _LLF
    if _LLF is None:
        _LLF = _autograd_function()
    return _LLF.apply(theta, windows, model, per_series)

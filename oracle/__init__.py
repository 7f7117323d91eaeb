"""FP64 oracle for the integrated / overlapping-exposure GP log-likelihood.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import this package.  It shares no code with
the CUDA path (``paper_2601_02527_gb300``) and neither imports the other.

Parts:
  * :func:`events` -- the event sequence of Section 3.2 (two events per
    exposure, one per instantaneous measurement, time-sorted; ties resolved
    end-before-start) and the slot of each exposure (instrument labels, or
    greedy interval colouring when none are given; footnote to Section
    3.2.3).
  * :func:`loglik` -- the sequential integrated Kalman filter in plain C,
    FP64, Van Loan discretisation (``gpss_oracle.c``), with complex-step
    gradients; :func:`exposure_grad`, :func:`condition` (integrated RTS
    smoother) and :func:`predict` (Algorithm 1) on the same model.
  * :mod:`oracle.dense` -- the dense integrated-GP log-likelihood
    (Section 2.1 with the integrated kernel of Section 3.1), used to pin the
    filter on small N.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgpss_oracle.so")
_lib = None

SHO = 1
MATERN32 = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math; FP64 throughout)."""
    src = os.path.join(_HERE, "gpss_oracle.c")
    hdr = os.path.join(_HERE, "oracle_body.h")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        lib.gpss_oracle_loglik.argtypes = [
            P(ctypes.c_int32), ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_int32),
            P(ctypes.c_int32), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
            P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
            P(ctypes.c_double)]
        lib.gpss_oracle_loglik.restype = ctypes.c_int
        lib.gpss_oracle_exposure_grad.argtypes = [
            P(ctypes.c_int32), ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_int32),
            P(ctypes.c_int32), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
            P(ctypes.c_double), ctypes.c_int64, P(ctypes.c_int64), P(ctypes.c_int64),
            P(ctypes.c_double), P(ctypes.c_double)]
        lib.gpss_oracle_exposure_grad.restype = ctypes.c_int
        lib.gpss_oracle_condition.argtypes = [
            P(ctypes.c_int32), ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_int32),
            P(ctypes.c_int32), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
            P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double)]
        lib.gpss_oracle_condition.restype = ctypes.c_int
        lib.gpss_oracle_predict.argtypes = [
            P(ctypes.c_int32), ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_int32),
            P(ctypes.c_int32), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
            P(ctypes.c_double), ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_double),
            P(ctypes.c_double)]
        lib.gpss_oracle_predict.restype = ctypes.c_int
        lib.gpss_oracle_discretize.argtypes = [
            P(ctypes.c_int32), P(ctypes.c_double), ctypes.c_double, P(ctypes.c_double),
            P(ctypes.c_double), P(ctypes.c_double)]
        lib.gpss_oracle_discretize.restype = ctypes.c_int
        lib.gpss_oracle_dim.argtypes = [P(ctypes.c_int32)]
        lib.gpss_oracle_dim.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def spec_array(terms, layout, n_slots, closed_form=False):
    """Model specification; ``closed_form`` selects the filter's timing mode
    (Appendix B closed forms for underdamped SHO terms, Van Loan otherwise)."""
    return np.asarray([len(terms), layout | (256 if closed_form else 0), n_slots] + list(terms),
                      dtype=np.int32)


def dim(terms, layout, n_slots) -> int:
    return _load().gpss_oracle_dim(_ptr(spec_array(terms, layout, n_slots), ctypes.c_int32))


class SelfOverlapError(ValueError):
    pass


def events(t_start, t_end, y, yerr, instrument=None):
    """Build the labelled event sequence of one series (Section 3.2.3).

    Returns a dict with per-event arrays ``t`` (float64), ``kind`` (0 start,
    1 end, 2 instantaneous measurement: t_start == t_end), ``slot`` (-1 for
    instantaneous), ``meas``, and for measurement events ``y``, ``r0`` (=
    yerr^2) and, at ends, ``invd`` (= 1/delta, delta = t_end - t_start in
    FP64), plus ``n_slots`` and ``n_meas``.

    Ordering: by time; at equal times every end comes before any start, so a
    reset never wipes an integral before it is read; then by measurement.
    Slots: the instrument label when given (each label must not overlap
    itself: t_end[n] <= t_start[next]); otherwise greedy interval colouring in
    start order, taking the lowest slot whose last exposure has ended.
    """
    t_start = np.asarray(t_start, np.float64)
    t_end = np.asarray(t_end, np.float64)
    n = len(t_start)
    delta = t_end - t_start
    if np.any(~np.isfinite(delta)) or np.any(delta < 0):
        raise ValueError("exposure lengths must be non-negative and finite")
    inst = delta == 0          # instantaneous measurements: one event, no slot
    integ = np.nonzero(~inst)[0]
    slot_of = np.full(n, -1, np.int64)
    if instrument is not None:
        lab = np.asarray(instrument, np.int64)
        if np.any(lab < 0):
            raise ValueError("instrument labels must be >= 0")
        slot_of[integ] = lab[integ]
        n_slots = int(lab[integ].max()) + 1 if len(integ) else 0
        for s in range(n_slots):
            idx = integ[lab[integ] == s]
            o = idx[np.argsort(t_start[idx], kind="stable")]
            if np.any(t_end[o[:-1]] > t_start[o[1:]]):
                raise SelfOverlapError(f"instrument {s} overlaps itself")
    else:
        last_end = []
        for i in integ[np.argsort(t_start[integ], kind="stable")]:
            for s, e in enumerate(last_end):
                if e <= t_start[i]:
                    slot_of[i] = s
                    last_end[s] = t_end[i]
                    break
            else:
                slot_of[i] = len(last_end)
                last_end.append(t_end[i])
        n_slots = len(last_end)
    ni = len(integ)
    ii = np.nonzero(inst)[0]
    t = np.concatenate([t_start[integ], t_end[integ], t_start[ii]])
    kind = np.concatenate([np.zeros(ni, np.int32), np.ones(ni, np.int32),
                           np.full(len(ii), 2, np.int32)])
    meas = np.concatenate([integ, integ, ii])
    # lexsort: last key is primary -> (time, ends then instants then starts,
    # measurement); same-time updates commute, a reset must follow the read
    korder = np.array([2, 0, 1])[kind]
    order = np.lexsort((meas, korder, t))
    t, kind, meas = t[order], kind[order], meas[order]
    y64 = np.asarray(y, np.float64)[meas]
    r0 = np.asarray(yerr, np.float64)[meas] ** 2
    with np.errstate(divide="ignore"):
        invd = np.where(kind == 1, 1.0 / np.where(kind == 1, delta[meas], 1.0), 0.0)
    obs = kind != 0
    return dict(t=t, kind=kind.astype(np.int32), slot=slot_of[meas].astype(np.int32), meas=meas,
                y=np.where(obs, y64, 0.0), r0=np.where(obs, r0, 0.0),
                invd=invd, n_slots=n_slots, n_meas=n)


def loglik_events(terms, layout, ev, theta, grad=False, n_slots=None, dump=False,
                  closed_form=False):
    """Oracle log-likelihood (and complex-step gradient) from built events.
    ``closed_form``: the timing mode (see spec_array); the parity reference is
    the default Van Loan discretisation."""
    lib = _load()
    n_slots = ev["n_slots"] if n_slots is None else n_slots
    spec = spec_array(terms, layout, n_slots, closed_form)
    theta = np.ascontiguousarray(theta, np.float64)
    out = np.zeros(1)
    g = np.zeros(len(theta)) if grad else None
    D = lib.gpss_oracle_dim(_ptr(spec, ctypes.c_int32))
    if D < 0:
        raise ValueError("unsupported model specification")
    n_ev = len(ev["t"])
    dP = np.zeros((n_ev, D, D)) if dump else None
    dS = np.zeros(int(np.sum(ev["kind"] != 0))) if dump else None
    arr = {k: np.ascontiguousarray(ev[k]) for k in ("t", "kind", "slot", "y", "r0", "invd")}
    rc = lib.gpss_oracle_loglik(
        _ptr(spec, ctypes.c_int32), n_ev, _ptr(arr["t"], ctypes.c_double),
        _ptr(arr["kind"], ctypes.c_int32), _ptr(arr["slot"], ctypes.c_int32),
        _ptr(arr["y"], ctypes.c_double), _ptr(arr["r0"], ctypes.c_double),
        _ptr(arr["invd"], ctypes.c_double), _ptr(theta, ctypes.c_double),
        _ptr(out, ctypes.c_double), _ptr(g, ctypes.c_double), _ptr(dP, ctypes.c_double),
        _ptr(dS, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle filter failed with code {rc}")
    res = {"loglik": float(out[0])}
    if grad:
        res["grad"] = g
    if dump:
        res["P"] = dP
        res["S"] = dS
    return res


def predict(terms, layout, t_start, t_end, y, yerr, theta, t_star, instrument=None,
            n_slots=None):
    """Oracle prediction of the latent f(t*) (mean, variance) given all of the
    series' data, at the test times t_star (Algorithm 1)."""
    ev = events(t_start, t_end, y, yerr, instrument)
    lib = _load()
    n_slots = ev["n_slots"] if n_slots is None else n_slots
    spec = spec_array(terms, layout, n_slots)
    theta = np.ascontiguousarray(theta, np.float64)
    ts = np.ascontiguousarray(t_star, np.float64)
    mean = np.zeros(len(ts))
    var = np.zeros(len(ts))
    arr = {k: np.ascontiguousarray(ev[k]) for k in ("t", "kind", "slot", "y", "r0", "invd")}
    rc = lib.gpss_oracle_predict(
        _ptr(spec, ctypes.c_int32), len(ev["t"]), _ptr(arr["t"], ctypes.c_double),
        _ptr(arr["kind"], ctypes.c_int32), _ptr(arr["slot"], ctypes.c_int32),
        _ptr(arr["y"], ctypes.c_double), _ptr(arr["r0"], ctypes.c_double),
        _ptr(arr["invd"], ctypes.c_double), _ptr(theta, ctypes.c_double), len(ts),
        _ptr(ts, ctypes.c_double), _ptr(mean, ctypes.c_double), _ptr(var, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle prediction failed with code {rc}")
    return mean, var


def exposure_grad_events(terms, layout, ev, theta, n_slots=None):
    """Complex-step d loglik / d t_start and d t_end per measurement (in the
    measurement order of the series) from built events."""
    lib = _load()
    n_slots = ev["n_slots"] if n_slots is None else n_slots
    spec = spec_array(terms, layout, n_slots)
    theta = np.ascontiguousarray(theta, np.float64)
    n_ev = len(ev["t"])
    n = ev["n_meas"]
    ks = np.zeros(n, np.int64)
    ke = np.zeros(n, np.int64)
    idx = np.arange(n_ev, dtype=np.int64)
    ks[ev["meas"][ev["kind"] == 0]] = idx[ev["kind"] == 0]
    ke[ev["meas"][ev["kind"] == 1]] = idx[ev["kind"] == 1]
    ks[ev["meas"][ev["kind"] == 2]] = idx[ev["kind"] == 2]
    ke[ev["meas"][ev["kind"] == 2]] = idx[ev["kind"] == 2]
    d_ts = np.zeros(n)
    d_te = np.zeros(n)
    arr = {k: np.ascontiguousarray(ev[k]) for k in ("t", "kind", "slot", "y", "r0", "invd")}
    rc = lib.gpss_oracle_exposure_grad(
        _ptr(spec, ctypes.c_int32), n_ev, _ptr(arr["t"], ctypes.c_double),
        _ptr(arr["kind"], ctypes.c_int32), _ptr(arr["slot"], ctypes.c_int32),
        _ptr(arr["y"], ctypes.c_double), _ptr(arr["r0"], ctypes.c_double),
        _ptr(arr["invd"], ctypes.c_double), _ptr(theta, ctypes.c_double), n,
        _ptr(ks, ctypes.c_int64), _ptr(ke, ctypes.c_int64), _ptr(d_ts, ctypes.c_double),
        _ptr(d_te, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle filter failed with code {rc}")
    return d_ts, d_te


def condition_events(terms, layout, ev, theta, n_slots=None):
    """Integrated RTS smoother (Eqs. rts, integrated_rts): conditioned mean
    and variance of every measurement's exposure average, in the series'
    measurement order."""
    lib = _load()
    n_slots = ev["n_slots"] if n_slots is None else n_slots
    spec = spec_array(terms, layout, n_slots)
    theta = np.ascontiguousarray(theta, np.float64)
    n_ev = len(ev["t"])
    me = np.zeros(n_ev)
    ve = np.zeros(n_ev)
    arr = {k: np.ascontiguousarray(ev[k]) for k in ("t", "kind", "slot", "y", "r0", "invd")}
    rc = lib.gpss_oracle_condition(
        _ptr(spec, ctypes.c_int32), n_ev, _ptr(arr["t"], ctypes.c_double),
        _ptr(arr["kind"], ctypes.c_int32), _ptr(arr["slot"], ctypes.c_int32),
        _ptr(arr["y"], ctypes.c_double), _ptr(arr["r0"], ctypes.c_double),
        _ptr(arr["invd"], ctypes.c_double), _ptr(theta, ctypes.c_double),
        _ptr(me, ctypes.c_double), _ptr(ve, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle smoother failed with code {rc}")
    n = ev["n_meas"]
    mean = np.zeros(n)
    var = np.zeros(n)
    end = ev["kind"] != 0
    mean[ev["meas"][end]] = me[end]
    var[ev["meas"][end]] = ve[end]
    return mean, var


def condition(terms, layout, t_start, t_end, y, yerr, theta, instrument=None, n_slots=None):
    """Oracle conditioned (mean, variance) of each measurement's exposure
    average given all the series' data."""
    ev = events(t_start, t_end, y, yerr, instrument)
    return condition_events(terms, layout, ev, theta, n_slots=n_slots)


def exposure_grad(terms, layout, t_start, t_end, y, yerr, theta, instrument=None, n_slots=None):
    """Oracle (d loglik / d t_start, d loglik / d t_end) of one series."""
    ev = events(t_start, t_end, y, yerr, instrument)
    return exposure_grad_events(terms, layout, ev, theta, n_slots=n_slots)


def loglik(terms, layout, t_start, t_end, y, yerr, theta, instrument=None, grad=False,
           n_slots=None, closed_form=False):
    """Oracle log-likelihood of one series; returns float or (float, grad)."""
    ev = events(t_start, t_end, y, yerr, instrument)
    r = loglik_events(terms, layout, ev, theta, grad=grad, n_slots=n_slots,
                      closed_form=closed_form)
    return (r["loglik"], r["grad"]) if grad else r["loglik"]


def discretize(terms, layout, n_slots, theta, dt, closed_form=False):
    """Phi~(dt), Q~(dt) and P0 of the augmented model (Van Loan + doubling, or
    with ``closed_form`` the Appendix B closed forms where they apply)."""
    lib = _load()
    spec = spec_array(terms, layout, n_slots, closed_form)
    D = lib.gpss_oracle_dim(_ptr(spec, ctypes.c_int32))
    Phi = np.zeros((D, D))
    Q = np.zeros((D, D))
    P0 = np.zeros((D, D))
    th = np.ascontiguousarray(theta, np.float64)
    rc = lib.gpss_oracle_discretize(_ptr(spec, ctypes.c_int32), _ptr(th, ctypes.c_double),
                                    float(dt), _ptr(Phi, ctypes.c_double),
                                    _ptr(Q, ctypes.c_double), _ptr(P0, ctypes.c_double))
    if rc:
        raise ValueError("unsupported model specification")
    return Phi, Q, P0


def _series_job(args):
    terms, layout, ser, th, grad = args[:5]
    closed_form = args[5] if len(args) > 5 else False
    ts, te, y, ye, inst = ser
    r = loglik(terms, layout, ts, te, y, ye, th, instrument=inst, grad=grad,
               closed_form=closed_form)
    return r


def loglik_workload(wl, series_idx=None, set_idx=None, grad=False, processes=1):
    """Oracle values for a ``synth.Workload``.

    With ``theta_per_series`` the result is indexed by series; otherwise by
    (set, series).  ``processes > 1`` uses a spawn-started pool.
    """
    if series_idx is None:
        series_idx = range(wl.n_series)
    jobs = []
    if wl.theta_per_series:
        for i in series_idx:
            jobs.append((wl.terms, wl.layout, wl.series(i), wl.theta[i], grad))
    else:
        sets = range(wl.theta.shape[0]) if set_idx is None else set_idx
        for s in sets:
            for i in series_idx:
                jobs.append((wl.terms, wl.layout, wl.series(i), wl.theta[s], grad))
    if processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            out = pool.map(_series_job, jobs)
    else:
        out = [_series_job(j) for j in jobs]
    if grad:
        return np.array([o[0] for o in out]), np.array([o[1] for o in out])
    return np.array(out)

"""Pins of the oracle's exposure-window gradient (complex step on the event
times, ``gpss_oracle_exposure_grad``).

  * against Richardson-extrapolated central differences of the dense
    integrated-GP log-likelihood (the plain definition, Section 3.1 with the
    closed-form double integral), which shares nothing with the filter: one
    SHO term, a sum of terms under both integral layouts, and overlapping
    exposures from two instruments;
  * time-shift invariance: moving every window by the same amount leaves the
    likelihood unchanged (stationary kernel), so the gradients sum to zero;
  * a measurement whose value does not enter (huge yerr) leaves the others'
    gradients as without it, up to its own small coupling.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import dense

SHO, M32 = 1, 2


def _fd(f, x, n, h):
    """Richardson-extrapolated central difference of f in coordinate n of x."""
    def c(hh):
        a = x.copy()
        b = x.copy()
        a[n] += hh
        b[n] -= hh
        return (f(a) - f(b)) / (2 * hh)
    return (4 * c(h / 2) - c(h)) / 3


def _check_against_dense(terms, layout, ts, te, y, ye, th, inst=None):
    d_ts, d_te = oracle.exposure_grad(terms, layout, ts, te, y, ye, th, instrument=inst)
    fd_ts = np.array([_fd(lambda a: dense.loglik(terms, th, a, te, y, ye), ts, n, 1e-4)
                      for n in range(len(ts))])
    fd_te = np.array([_fd(lambda a: dense.loglik(terms, th, ts, a, y, ye), te, n, 1e-4)
                      for n in range(len(ts))])
    for got, ref in ((d_ts, fd_ts), (d_te, fd_te)):
        assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref) + 1e-7 * np.abs(ref).max()), (got, ref)
    return d_ts, d_te


def _series(rng, n):
    ts, te = synth.single_instrument_exposures(rng, n, 1.0, 0.05, 0.5)
    # keep a little dead time so central differences never cross an event tie
    te = np.minimum(te, np.append(ts[1:] - 1e-3, np.inf))
    return ts, te


def test_single_sho_matches_dense(oracle_lib):
    rng = np.random.default_rng(11)
    ts, te = _series(rng, 30)
    y = rng.normal(size=30)
    ye = np.full(30, 0.05)
    _check_against_dense([SHO], 0, ts, te, y, ye, np.array([1.0, 2 * math.pi / 5, 3.0, 0.1]))


@pytest.mark.parametrize("layout", [0, 1])
def test_sum_of_terms_matches_dense(oracle_lib, layout):
    rng = np.random.default_rng(12)
    ts, te = _series(rng, 24)
    y = rng.normal(size=24)
    ye = np.full(24, 0.1)
    th = np.array([1.0, 0.9, 4.0, 0.5, 3.0, 0.7, 0.1])
    _check_against_dense([SHO, SHO], layout, ts, te, y, ye, th)


def test_overlapping_instruments_match_dense(oracle_lib):
    rng = np.random.default_rng(13)
    a = np.sort(rng.uniform(0, 30, 14))
    b = np.sort(rng.uniform(0, 30, 10))
    ts = np.concatenate([a, b])
    te = np.concatenate([np.minimum(a + rng.uniform(0.2, 1.5, 14), np.append(a[1:] - 1e-3, 99)),
                         np.minimum(b + rng.uniform(0.5, 2.5, 10), np.append(b[1:] - 1e-3, 99))])
    inst = np.concatenate([np.zeros(14, np.int32), np.ones(10, np.int32)])
    y = rng.normal(size=24)
    ye = np.full(24, 0.08)
    th = np.array([1.0, 1.3, 2.0, 0.6, 4.0, 0.1])
    _check_against_dense([SHO, M32], 0, ts, te, y, ye, th, inst=inst)


def test_time_shift_invariance(oracle_lib):
    rng = np.random.default_rng(14)
    ts, te = synth.single_instrument_exposures(rng, 60, 1.0, 0.05, 0.5)
    y = rng.normal(size=60)
    ye = np.full(60, 0.05)
    th = np.array([1.0, 2.0, 1.5, 0.3, 5.0, 0.1])
    d_ts, d_te = oracle.exposure_grad([SHO, M32], 0, ts, te, y, ye, th)
    scale = np.abs(np.concatenate([d_ts, d_te])).sum()
    assert abs(d_ts.sum() + d_te.sum()) <= 1e-11 * scale

"""Pins of the oracle's prediction at arbitrary times (``gpss_oracle_predict``,
Algorithm 1 on the augmented model): mean and variance of the latent f(t*)
given all of the series' exposure-averaged data.

  * against the dense GP prediction, the plain definition (k*^T (K + R)^-1 y,
    k(0) - k*^T (K + R)^-1 k*, k*_n the covariance of f(t*) with the n-th
    exposure average through the kernel's first antiderivative): test times
    before the data (retrodiction), at the first event, on every event time,
    inside exposures and gaps, after the data (extrapolation); one SHO term,
    sums under both integral layouts, overlapping instruments;
  * far from the data the prediction returns to the prior (mean 0,
    variance k(0)).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import dense

SHO, M32 = 1, 2


def _grid(ts, te, rng):
    inside = ts + rng.uniform(0, 1, len(ts)) * (te - ts)
    return np.concatenate([[ts[0] - 3.0, ts[0] - 0.2, ts[0]], ts, te, inside,
                           np.linspace(ts[0], te[-1], 41), [te[-1] + 0.5, te[-1] + 4.0]])


def _check(terms, layout, ts, te, y, ye, th, tq, inst=None):
    mu, va = oracle.predict(terms, layout, ts, te, y, ye, th, tq, instrument=inst)
    mu_d, va_d = dense.predict(terms, th, ts, te, y, ye, tq)
    assert np.max(np.abs(mu - mu_d)) <= 1e-9 * np.abs(mu_d).max(), (mu, mu_d)
    assert np.all(np.abs(va - va_d) <= 1e-7 * va_d + 1e-12), (va, va_d)


def test_single_sho(oracle_lib):
    rng = np.random.default_rng(31)
    ts, te = synth.single_instrument_exposures(rng, 40, 1.0, 0.05, 0.5)
    y = rng.normal(size=40)
    _check([SHO], 0, ts, te, y, np.full(40, 0.05), np.array([1.0, 2 * math.pi / 5, 3.0, 0.1]),
           _grid(ts, te, rng))


@pytest.mark.parametrize("layout", [0, 1])
def test_sum_of_terms(oracle_lib, layout):
    rng = np.random.default_rng(32)
    ts, te = synth.single_instrument_exposures(rng, 35, 1.0, 0.05, 0.5)
    y = rng.normal(size=35)
    th = np.array([1.0, 0.9, 4.0, 0.5, 3.0, 0.7, 0.1])
    _check([SHO, SHO], layout, ts, te, y, np.full(35, 0.1), th, _grid(ts, te, rng))


def test_overlapping_instruments(oracle_lib):
    rng = np.random.default_rng(33)
    a = np.sort(rng.uniform(0, 30, 16))
    b = np.sort(rng.uniform(0.05, 30, 12))
    ts = np.concatenate([a, b])
    te = np.concatenate([np.minimum(a + rng.uniform(0.2, 1.5, 16), np.append(a[1:] - 1e-3, 99)),
                         np.minimum(b + rng.uniform(0.5, 2.5, 12), np.append(b[1:] - 1e-3, 99))])
    inst = np.concatenate([np.zeros(16, np.int32), np.ones(12, np.int32)])
    y = rng.normal(size=28)
    th = np.array([1.0, 1.3, 2.0, 0.6, 4.0, 0.1])
    o = np.argsort(ts, kind="stable")
    tq = _grid(ts[o], te[o], rng)
    _check([SHO, M32], 0, ts, te, y, np.full(28, 0.08), th, tq, inst=inst)


def test_prior_far_away(oracle_lib):
    rng = np.random.default_rng(34)
    ts, te = synth.single_instrument_exposures(rng, 20, 1.0, 0.05, 0.5)
    y = rng.normal(size=20)
    th = np.array([1.3, 2.0, 3.0, 0.1])
    mu, va = oracle.predict([SHO], 0, ts, te, y, np.full(20, 0.05), th,
                            [ts[0] - 500.0, te[-1] + 500.0])
    assert np.all(np.abs(mu) <= 1e-12) and np.allclose(va, 1.3 ** 2, rtol=1e-12)

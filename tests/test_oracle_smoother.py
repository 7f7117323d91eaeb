"""Pins of the oracle's integrated RTS smoother (``gpss_oracle_condition``,
Eqs. rts and integrated_rts): the conditioned mean and variance of every
measurement's exposure average given all the data.

  * against the dense integrated-GP posterior, the plain definition
    (mean K (K + R)^-1 y, variance diag(K - K (K + R)^-1 K) with K the
    integrated kernel of the exposure averages), which shares nothing with
    the filter: one SHO term, sums under both integral layouts, overlapping
    instruments (several integral slots) and unlabelled overlaps;
  * the posterior variance lies in (0, prior variance];
  * a measurement with a huge error bar barely moves the others' means.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import dense

SHO, M32 = 1, 2


def _dense_posterior(terms, th, ts, te, y, ye):
    _, s = dense.split_theta(terms, th)
    K = dense.integrated_cov(terms, th, ts, te)
    A = K + np.diag(np.asarray(ye) ** 2 + s * s)
    return K @ np.linalg.solve(A, y), np.diag(K - K @ np.linalg.solve(A, K)), np.diag(K)


def _check(terms, layout, ts, te, y, ye, th, inst=None):
    mu, va = oracle.condition(terms, layout, ts, te, y, ye, th, instrument=inst)
    mu_d, va_d, prior = _dense_posterior(terms, th, ts, te, y, ye)
    assert np.max(np.abs(mu - mu_d)) <= 1e-9 * np.max(np.abs(mu_d)), (mu, mu_d)
    # the posterior variance is a difference of prior-sized terms on both
    # sides (about 60x the result here), so a few digits go
    assert np.all(np.abs(va - va_d) <= 1e-7 * va_d), (va, va_d)
    assert np.all(va > 0) and np.all(va <= prior * (1 + 1e-12))
    return mu, va


def test_single_sho(oracle_lib):
    rng = np.random.default_rng(21)
    ts, te = synth.single_instrument_exposures(rng, 60, 1.0, 0.05, 0.5)
    y = rng.normal(size=60)
    _check([SHO], 0, ts, te, y, np.full(60, 0.05), np.array([1.0, 2 * math.pi / 5, 3.0, 0.1]))


@pytest.mark.parametrize("layout", [0, 1])
def test_sum_of_terms(oracle_lib, layout):
    rng = np.random.default_rng(22)
    ts, te = synth.single_instrument_exposures(rng, 50, 1.0, 0.05, 0.5)
    y = rng.normal(size=50)
    th = np.array([1.0, 0.9, 4.0, 0.5, 3.0, 0.7, 0.1])
    _check([SHO, SHO], layout, ts, te, y, np.full(50, 0.1), th)


def test_overlapping_instruments(oracle_lib):
    rng = np.random.default_rng(23)
    a = np.sort(rng.uniform(0, 40, 20))
    b = np.sort(rng.uniform(0, 40, 15))
    ts = np.concatenate([a, b])
    te = np.concatenate([np.minimum(a + rng.uniform(0.2, 1.5, 20), np.append(a[1:], 99)),
                         np.minimum(b + rng.uniform(0.5, 2.5, 15), np.append(b[1:], 99))])
    inst = np.concatenate([np.zeros(20, np.int32), np.ones(15, np.int32)])
    y = rng.normal(size=35)
    th = np.array([1.0, 1.3, 2.0, 0.6, 4.0, 0.1])
    _check([SHO, M32], 0, ts, te, y, np.full(35, 0.08), th, inst=inst)


def test_three_open_unlabelled(oracle_lib):
    rng = np.random.default_rng(24)
    ts, te, _ = synth.capped_overlap_exposures(rng, 45, 0.5, 0.5, 3.0, cap=3)
    y = rng.normal(size=45)
    _check([SHO], 0, ts, te, y, np.full(45, 0.1), np.array([1.0, 2 * math.pi / 10, 3.0, 0.1]))


def test_uninformative_point(oracle_lib):
    # a measurement with a huge error bar conditions the others like a
    # series without it
    rng = np.random.default_rng(25)
    ts, te = synth.single_instrument_exposures(rng, 30, 1.0, 0.05, 0.5)
    y = rng.normal(size=30)
    ye = np.full(30, 0.05)
    th = np.array([1.0, 2.0, 3.0, 0.1])
    ye[12], y[12] = 1e6, 50.0
    mu, va = oracle.condition([SHO], 0, ts, te, y, ye, th)
    keep = np.arange(30) != 12
    mu0, va0 = oracle.condition([SHO], 0, ts[keep], te[keep], y[keep], ye[keep], th)
    assert np.max(np.abs(mu[keep] - mu0)) <= 1e-9 * np.max(np.abs(mu0))
    assert np.max(np.abs(va[keep] - va0) / va0) <= 1e-8


def test_touching_windows(oracle_lib):
    # each exposure ends exactly where the next starts (end before start)
    rng = np.random.default_rng(26)
    ts = np.arange(70) * 0.5
    _check([SHO], 0, ts, ts + 0.5, rng.normal(size=70), np.full(70, 0.05),
           np.array([1.0, 2 * math.pi / 10, 3.0, 0.1]))

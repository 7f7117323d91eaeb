"""Pins for instantaneous measurements (t_start == t_end) in the oracles.

An instantaneous measurement observes the latent f(t) = H x(t) directly
(Section 2: the plain SSM with H = (1 0 1 0 ...)); it is the delta -> 0 limit
of an exposure average (Section 3.2).  A series may mix both kinds.  Pinned:

  * pure instantaneous series against the dense GP with K_ij = k(|t_i - t_j|)
    (the plain definition, built from the kernel alone);
  * the dense cross-covariance of an instant with an exposure against
    quadrature of the kernel;
  * mixed series against the dense GP (sums of terms, overdamped terms, an
    instant coinciding with an exposure start or end);
  * the integrated oracle converging to the instantaneous one as every
    exposure shrinks around its instant, at O(delta^2);
  * the complex-step gradient against central differences, the derivative
    with respect to an instant's time against central differences, and the
    smoother and the prediction against the dense posterior and prediction.
"""
import math

import numpy as np
import pytest
import scipy.integrate

import oracle
import synth
from oracle import dense

SHO, M32 = 1, 2


def _signal(rng, ts, te, terms, th):
    return synth.exposure_average_signal(rng, ts, te, terms, np.asarray(th, float))


def _instants(seed, n, gap=0.7):
    rng = np.random.default_rng(seed)
    return rng, np.cumsum(rng.exponential(gap, n))


@pytest.mark.parametrize("terms,theta", [([SHO], [1.0, 2 * math.pi / 10, 3.0, 0.1]),
                                         ([SHO, M32], [1.0, 1.1, 2.0, 0.5, 4.0, 0.15]),
                                         ([SHO], [0.8, 1.3, 0.2, 0.1])])
def test_pure_instantaneous_matches_dense(oracle_lib, terms, theta):
    rng, t = _instants(81, 300)
    y = rng.standard_normal(len(t))
    ye = np.full(len(t), 0.05)
    lk = oracle.loglik(terms, 0, t, t, y, ye, theta)
    K = dense.instantaneous_cov(terms, theta, t)
    ld = dense.gaussian_loglik(K, y, ye ** 2 + theta[-1] ** 2)
    assert abs(lk - ld) <= 1e-9 * abs(ld), (lk, ld)
    assert oracle.events(t, t, y, ye)["n_slots"] == 0


@pytest.mark.parametrize("q", [0.3, 3.0])
def test_dense_cross_covariance_matches_quadrature(q):
    sig, w0 = 1.1, 0.9
    for t, (a, b) in ((0.3, (0.0, 1.0)), (2.5, (0.2, 1.4)), (-1.0, (0.0, 2.0)), (1.0, (1.0, 3.0))):
        ref, _ = scipy.integrate.quad(lambda s: dense.kernel(t - s, sig, w0, q), a, b,
                                      points=[t] if a < t < b else None, epsabs=1e-14,
                                      epsrel=1e-13)
        K = dense.integrated_cov([SHO], [sig, w0, q, 0.1], np.array([t, a]), np.array([t, b]))
        assert abs(K[0, 1] - ref / (b - a)) <= 1e-11, (t, K[0, 1], ref / (b - a))
        assert abs(K[0, 0] - sig ** 2) <= 1e-14


def _mixed(seed, n, terms, th, coincide=True):
    rng = np.random.default_rng(seed)
    ts, te = synth.single_instrument_exposures(rng, n, 1.0, 0.05, 0.5)
    inst = np.sort(rng.uniform(ts[0] - 1.0, te[-1] + 1.0, n // 2))
    if coincide:
        inst[:3] = [ts[5], te[7], ts[9]]  # an instant at an exposure's start / end
    a = np.concatenate([ts, inst])
    b = np.concatenate([te, inst])
    y = _signal(rng, a, np.where(b > a, b, a + 1e-9), terms, th) + 0.1 * rng.standard_normal(len(a))
    ye = np.full(len(a), 0.02)
    return a, b, y, ye


@pytest.mark.parametrize("terms,layout,theta", [([SHO], 0, [1.0, 0.7, 3.0, 0.1]),
                                                ([SHO, M32], 0, [1.0, 1.1, 2.0, 0.5, 3.0, 0.1]),
                                                ([SHO, SHO], 1, [1.0, 0.7, 3.0, 0.5, 2.0, 0.3, 0.1])])
def test_mixed_series_matches_dense(oracle_lib, terms, layout, theta):
    a, b, y, ye = _mixed(82, 160, terms, theta)
    lk = oracle.loglik(terms, layout, a, b, y, ye, theta)
    ld = dense.loglik(terms, theta, a, b, y, ye)
    assert abs(lk - ld) <= 1e-9 * abs(ld), (lk, ld)


def test_integrated_converges_to_instantaneous(oracle_lib):
    th = [1.0, 2 * math.pi / 10, 3.0, 0.1]
    rng, t = _instants(83, 120, gap=1.0)
    y = rng.standard_normal(len(t))
    ye = np.zeros(len(t))
    l_inst = oracle.loglik([SHO], 0, t, t, y, ye, th)
    gaps = []
    for d in (0.08, 0.04, 0.02, 0.01):
        gaps.append(oracle.loglik([SHO], 0, t - d / 2, t + d / 2, y, ye, th) - l_inst)
    r = [gaps[i] / gaps[i + 1] for i in range(3)]
    assert all(3.6 < x < 4.4 for x in r), (gaps, r)


def test_gradients(oracle_lib):
    terms, th = [SHO, M32], np.array([1.0, 1.1, 2.0, 0.5, 3.0, 0.1])
    a, b, y, ye = _mixed(84, 60, terms, th)
    l0, g = oracle.loglik(terms, 0, a, b, y, ye, th, grad=True)
    for i in range(len(th)):
        h = 1e-4 * th[i]
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (oracle.loglik(terms, 0, a, b, y, ye, tp) - oracle.loglik(terms, 0, a, b, y, ye, tm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-2 * abs(l0)), (i, fd, g[i])
    d_ts, d_te = oracle.exposure_grad(terms, 0, a, b, y, ye, th)
    inst = np.nonzero(a == b)[0]
    np.testing.assert_array_equal(d_ts[inst], d_te[inst])
    for n in inst[3:9]:
        h = 1e-6
        ap, am = a.copy(), a.copy()
        ap[n] += h
        am[n] -= h
        fd = (oracle.loglik(terms, 0, ap, ap * (a == b) + b * (a != b), y, ye, th) -
              oracle.loglik(terms, 0, am, am * (a == b) + b * (a != b), y, ye, th)) / (2 * h)
        assert abs(fd - (d_ts[n] + d_te[n])) <= 1e-6 * max(1.0, abs(fd)), (n, fd, d_ts[n])


def test_smoother_and_prediction_match_dense(oracle_lib):
    terms, th = [SHO, M32], [1.0, 1.1, 2.0, 0.5, 3.0, 0.1]
    a, b, y, ye = _mixed(85, 100, terms, th)
    mu, va = oracle.condition(terms, 0, a, b, y, ye, th)
    mu_d, va_d = dense.posterior(terms, th, a, b, y, ye)
    assert np.max(np.abs(mu - mu_d)) <= 1e-9 * np.abs(mu_d).max()
    assert np.all(np.abs(va - va_d) <= 1e-7 * va_d + 1e-12)
    tq = np.concatenate([[a.min() - 1.0], a, b, np.linspace(a.min(), b.max(), 50), [b.max() + 2]])
    mu, va = oracle.predict(terms, 0, a, b, y, ye, th, tq)
    mu_d, va_d = dense.predict(terms, th, a, b, y, ye, tq)
    assert np.max(np.abs(mu - mu_d)) <= 1e-9 * np.abs(mu_d).max()
    assert np.all(np.abs(va - va_d) <= 1e-7 * va_d + 1e-12)

"""Pins for the overdamped SHO (Q < 1/2) in the oracles.

Appendix B prints the transition matrix of the overdamped oscillator (cosh and
sinh in place of cos and sin) but none of its noise or integral blocks; the
oracle's Van Loan discretisation covers every Q > 0 without a special case,
and the dense oracle writes the kernel as two real exponentials.  Pinned here:

  * the dense kernel against the stationary covariance of the oscillator's
    SDE, k(tau) = [exp(F tau) P_inf]_00 (Section 2.2), by a library matrix
    exponential, and its continuity at Q -> 1/2 (the Matern-3/2 limit);
  * the dense integrated covariance and the first antiderivative against
    numerical quadrature of that kernel;
  * the filter oracle against the dense log-likelihood (one term, sums with a
    Matern-3/2 or a second SHO under both integral layouts, overlapping
    instruments);
  * its complex-step gradient against central differences;
  * the smoother and the prediction against the dense posterior and the dense
    prediction.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle
import synth
from oracle import dense

SHO, M32 = 1, 2


@pytest.mark.parametrize("q", [0.02, 0.1, 0.3, 0.49])
def test_kernel_is_the_sde_covariance(q):
    sigma, w0 = 1.3, 0.8
    F = np.array([[0.0, 1.0], [-w0 * w0, -w0 / q]])
    Pinf = sigma ** 2 * np.diag([1.0, w0 * w0])
    for tau in (0.0, 1e-3, 0.1, 1.0, 4.0, 30.0, 300.0):
        ref = (scipy.linalg.expm(F * tau) @ Pinf)[0, 0]
        got = dense.kernel(tau, sigma, w0, q)
        assert abs(got - ref) <= 1e-12 * sigma ** 2 + 1e-10 * abs(ref), (tau, got, ref)


def test_kernel_continuous_at_critical_damping():
    x = np.linspace(0, 20, 201)
    m = dense.kernel(x, 1.0, 1.1, 0.5)
    assert np.max(np.abs(dense.kernel(x, 1.0, 1.1, 0.5 - 1e-7) - m)) <= 1e-6
    assert np.max(np.abs(dense.kernel(x, 1.0, 1.1, 0.5 + 1e-7) - m)) <= 1e-6


@pytest.mark.parametrize("q", [0.08, 0.35])
@pytest.mark.parametrize("win", [((0.0, 1.0), (0.4, 2.9)), ((0.0, 3.0), (1.0, 1.5)),
                                 ((0.0, 0.7), (2.2, 2.5)), ((0.0, 1.0), (1.0, 2.0))])
def test_integrated_cov_matches_quadrature(q, win):
    (a1, b1), (a2, b2) = win
    sigma, w0 = 0.9, 1.7
    pts = sorted({a1, b1, a2, b2})
    ref = 0.0
    for lo, hi in zip(pts[:-1], pts[1:]):
        if lo < a1 or hi > b1:
            continue
        v, _ = scipy.integrate.dblquad(lambda tp, t: dense.kernel(t - tp, sigma, w0, q),
                                       lo, hi, a2, b2, epsabs=1e-13, epsrel=1e-12)
        ref += v
    ref /= (b1 - a1) * (b2 - a2)
    K = dense.integrated_cov([SHO], [sigma, w0, q, 0.1], np.array([a1, a2]), np.array([b1, b2]))
    assert abs(K[0, 1] - ref) <= 1e-9 * abs(ref), (K[0, 1], ref)


@pytest.mark.parametrize("q", [0.08, 0.35])
def test_first_antiderivative_matches_quadrature(q):
    for x in (-4.0, -0.3, 0.2, 1.0, 7.5):
        ref, _ = scipy.integrate.quad(lambda u: dense.kernel(u, 1.2, 0.9, q), 0.0, x,
                                      epsabs=1e-14, epsrel=1e-13)
        assert abs(dense.F1(x, 1.2, 0.9, q) - ref) <= 1e-11, (x, ref)


def _check_dense(terms, layout, ts, te, y, ye, th, inst=None):
    lk = oracle.loglik(terms, layout, ts, te, y, ye, th, instrument=inst)
    ld = dense.loglik(terms, th, ts, te, y, ye)
    assert abs(lk - ld) <= 1e-9 * abs(ld), (lk, ld)
    return lk


@pytest.mark.parametrize("q", [0.05, 0.2, 0.45])
def test_filter_matches_dense_single_term(oracle_lib, q):
    th = [1.0, 2 * math.pi / 10, q, 0.1]
    wl = synth.small_single(61, 250, [SHO], th)
    ts, te, y, ye, _ = wl.series(0)
    _check_dense([SHO], 0, ts, te, y, ye, wl.theta[0])


def test_filter_matches_dense_sums_and_layouts(oracle_lib):
    th = [1.0, 1.5, 0.2, 0.5, 4.0, 0.1]
    wl = synth.small_single(62, 200, [SHO, M32], th)
    ts, te, y, ye, _ = wl.series(0)
    _check_dense([SHO, M32], 0, ts, te, y, ye, wl.theta[0])
    th2 = [1.0, 0.7, 3.0, 0.5, 2.0, 0.3, 0.1]
    wl = synth.small_single(63, 200, [SHO, SHO], th2)
    ts, te, y, ye, _ = wl.series(0)
    a = _check_dense([SHO, SHO], 0, ts, te, y, ye, wl.theta[0])
    b = _check_dense([SHO, SHO], 1, ts, te, y, ye, wl.theta[0])
    assert abs(a - b) <= 1e-12 * abs(a)


def test_filter_matches_dense_overlapping_instruments(oracle_lib):
    rng = np.random.default_rng(64)
    a = np.sort(rng.uniform(0, 80, 60))
    b = np.sort(rng.uniform(0.03, 80, 40))
    ts = np.concatenate([a, b])
    te = np.concatenate([np.minimum(a + rng.uniform(0.2, 1.5, 60), np.append(a[1:], 99.0)),
                         np.minimum(b + rng.uniform(0.5, 3.0, 40), np.append(b[1:], 99.0))])
    inst = np.concatenate([np.zeros(60, np.int32), np.ones(40, np.int32)])
    th = np.array([0.8, 1.1, 0.25, 0.6, 3.0, 0.15])
    sig = synth.exposure_average_signal(rng, ts, te, [SHO, M32], th)
    y = sig + 0.15 * rng.standard_normal(len(ts))
    ye = np.zeros(len(ts))
    _check_dense([SHO, M32], 0, ts, te, y, ye, th, inst=inst)


@pytest.mark.parametrize("terms,layout,theta", [
    ([SHO], 0, [1.0, 0.9, 0.3, 0.1]),
    ([SHO, M32], 0, [1.0, 0.8, 0.12, 0.5, 4.0, 0.15]),
    ([SHO, SHO], 1, [1.0, 0.7, 3.0, 0.5, 3.0, 0.4, 0.1])])
def test_complex_step_gradient(oracle_lib, terms, layout, theta):
    wl = synth.small_single(65, 120, terms, theta)
    ts, te, y, ye, _ = wl.series(0)
    th = np.asarray(theta, float)
    l0, g = oracle.loglik(terms, layout, ts, te, y, ye, th, grad=True)

    def central(i, h):
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        return (oracle.loglik(terms, layout, ts, te, y, ye, tp)
                - oracle.loglik(terms, layout, ts, te, y, ye, tm)) / (2 * h)

    for i in range(len(th)):
        h = 1e-3 * th[i]
        fd = (4 * central(i, h / 2) - central(i, h)) / 3
        assert abs(fd - g[i]) <= 1e-7 * max(abs(g[i]), 1e-2 * abs(l0)), (i, fd, g[i])


def test_smoother_and_prediction_match_dense(oracle_lib):
    th = [1.0, 1.2, 0.15, 0.1]
    wl = synth.small_single(66, 150, [SHO], th)
    ts, te, y, ye, _ = wl.series(0)
    mu, va = oracle.condition([SHO], 0, ts, te, y, ye, wl.theta[0])
    mu_d, va_d = dense.posterior([SHO], wl.theta[0], ts, te, y, ye)
    assert np.max(np.abs(mu - mu_d)) <= 1e-9 * np.abs(mu_d).max()
    assert np.all(np.abs(va - va_d) <= 1e-7 * va_d + 1e-12)
    rng = np.random.default_rng(67)
    tq = np.concatenate([[ts[0] - 2.0], ts, te, ts + rng.uniform(0, 1, len(ts)) * (te - ts),
                         [te[-1] + 1.0]])
    mu, va = oracle.predict([SHO], 0, ts, te, y, ye, wl.theta[0], tq)
    mu_d, va_d = dense.predict([SHO], wl.theta[0], ts, te, y, ye, tq)
    assert np.max(np.abs(mu - mu_d)) <= 1e-9 * np.abs(mu_d).max()
    assert np.all(np.abs(va - va_d) <= 1e-7 * va_d + 1e-12)

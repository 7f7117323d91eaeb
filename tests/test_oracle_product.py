"""Pins for product kernels (Appendix C.2) in the oracles.

A product of two SHO terms, k = sigma^2 k_a k_b (unit-variance factors,
parameters (sigma, omega_a, Q_a, omega_b, Q_b)), is the SSM with
F = F_a (x) I + I (x) F_b, P_inf = P_inf,a (x) P_inf,b and observation
H = H_a (x) H_b (the first component).  Pinned:

  * the observed stationary covariance [exp(F tau) P_inf]_00 of the oracle's
    product model against the plain product of the two kernels;
  * the oracle's Van Loan Q of the product against Eq. product_Q built from
    the two single-oscillator discretisations;
  * log-likelihoods of instantaneous series (a product alone, and summed with
    an SHO) against the dense GP of the product kernel, and of a small
    integrated series (exposure averages, two overlapping instruments)
    against the dense GP by quadrature of the kernel;
  * the complex-step gradient against central differences, and the
    smoother and the prediction against the dense posterior and prediction.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import dense

SHO, M32, PROD = 1, 2, 3


def test_product_covariance_and_noise(oracle_lib):
    sig, wa, qa, wb, qb = 1.3, 0.4, 5.0, 2.1, 0.8
    th = [sig, wa, qa, wb, qb, 0.1]
    p = (sig, wa, qa, wb, qb)
    _, _, P0 = oracle.discretize([PROD], 0, 0, th, 0.0)
    for tau in (0.0, 0.05, 0.7, 3.0, 11.0):
        Phi, Q, _ = oracle.discretize([PROD], 0, 0, th, tau)
        assert abs((Phi @ P0)[0, 0] - dense.term_kernel(tau, p)) <= 1e-12 * sig ** 2
        # Eq. product_Q from the factors' own discretisations
        _, Qa, Pa = oracle.discretize([SHO], 0, 0, [1.0, wa, qa, 0.1], tau)
        _, Qb, Pb = oracle.discretize([SHO], 0, 0, [sig, wb, qb, 0.1], tau)
        ref = np.kron(Pa, Qb) + np.kron(Qa, Pb) - np.kron(Qa, Qb)
        assert np.max(np.abs(Q - ref)) <= 1e-12 * np.max(np.abs(P0)), (tau, Q, ref)


def _inst(seed, n):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(0.6, n))
    return rng, t, rng.standard_normal(n), np.full(n, 0.05)


@pytest.mark.parametrize("terms,theta", [([PROD], [1.0, 0.3, 4.0, 1.7, 1.5, 0.1]),
                                         ([PROD, SHO], [1.0, 0.3, 4.0, 1.7, 0.4, 0.5, 2.5, 3.0, 0.1])])
def test_instantaneous_matches_dense(oracle_lib, terms, theta):
    _, t, y, ye = _inst(101, 250)
    lk = oracle.loglik(terms, 0, t, t, y, ye, theta)
    ld = dense.gaussian_loglik(dense.instantaneous_cov(terms, theta, t), y, ye ** 2 + theta[-1] ** 2)
    assert abs(lk - ld) <= 1e-9 * abs(ld), (lk, ld)


def test_integrated_matches_quadrature(oracle_lib):
    th = [1.0, 0.5, 3.0, 1.9, 2.0, 0.1]
    ts = np.array([0.0, 0.8, 1.9, 3.1, 4.0, 5.2])
    te = ts + np.array([0.5, 0.6, 0.9, 0.4, 1.0, 0.3])
    t2 = np.array([0.3, 2.2, 4.4])
    a = np.concatenate([ts, t2])
    b = np.concatenate([te, t2 + 1.5])
    inst = np.array([0] * 6 + [1] * 3, np.int32)
    rng = np.random.default_rng(102)
    y = rng.standard_normal(len(a))
    ye = np.full(len(a), 0.1)
    lk = oracle.loglik([PROD], 0, a, b, y, ye, th, instrument=inst)
    ld = dense.loglik([PROD], th, a, b, y, ye)
    assert abs(lk - ld) <= 1e-8 * abs(ld), (lk, ld)


def test_gradient(oracle_lib):
    terms, th = [PROD, SHO], np.array([1.0, 0.3, 4.0, 1.7, 0.4, 0.5, 2.5, 3.0, 0.1])
    _, t, y, ye = _inst(103, 80)
    l0, g = oracle.loglik(terms, 0, t, t, y, ye, th, grad=True)
    for i in range(len(th)):
        h = 1e-4 * th[i]
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (oracle.loglik(terms, 0, t, t, y, ye, tp) - oracle.loglik(terms, 0, t, t, y, ye, tm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-2 * abs(l0)), (i, fd, g[i])


def test_smoother_and_prediction(oracle_lib):
    terms, th = [PROD], [1.0, 0.3, 4.0, 1.7, 1.5, 0.1]
    _, t, y, ye = _inst(104, 120)
    mu, va = oracle.condition(terms, 0, t, t, y, ye, th)
    mu_d, va_d = dense.posterior(terms, th, t, t, y, ye)
    assert np.max(np.abs(mu - mu_d)) <= 1e-9 * np.abs(mu_d).max()
    assert np.all(np.abs(va - va_d) <= 1e-7 * va_d + 1e-12)
    tq = np.concatenate([[t[0] - 1.0], t[::3], np.linspace(t[0], t[-1], 40), [t[-1] + 1.5]])
    mu, va = oracle.predict(terms, 0, t, t, y, ye, th, tq)
    mu_d, va_d = dense.predict(terms, th, t, t, y, ye, tq)
    assert np.max(np.abs(mu - mu_d)) <= 1e-9 * np.abs(mu_d).max()
    assert np.all(np.abs(va - va_d) <= 1e-7 * va_d + 1e-12)


def test_integrated_smoother_and_prediction(oracle_lib):
    # exposure averages with a product kernel (two overlapping instruments):
    # the oracle's integrated RTS smoother and Algorithm 1 prediction against
    # the dense posterior and prediction (kernel integrals by quadrature)
    th = [1.0, 0.5, 3.0, 1.9, 2.0, 0.1]
    ts = np.array([0.0, 0.8, 1.9, 3.1, 4.0])
    te = ts + np.array([0.5, 0.6, 0.9, 0.4, 1.0])
    t2 = np.array([0.3, 2.2])
    a = np.concatenate([ts, t2])
    b = np.concatenate([te, t2 + 1.5])
    inst = np.array([0] * 5 + [1] * 2, np.int32)
    rng = np.random.default_rng(105)
    y = rng.standard_normal(len(a))
    ye = np.full(len(a), 0.1)
    mu, va = oracle.condition([PROD], 0, a, b, y, ye, th, instrument=inst)
    mu_d, va_d = dense.posterior([PROD], th, a, b, y, ye)
    assert np.max(np.abs(mu - mu_d)) <= 1e-8 * np.abs(mu_d).max()
    assert np.all(np.abs(va - va_d) <= 1e-7 * va_d + 1e-11)
    tq = np.array([-0.5, 0.2, 1.0, 2.5, 4.6, 6.0])
    mu, va = oracle.predict([PROD], 0, a, b, y, ye, th, tq, instrument=inst)
    mu_d, va_d = dense.predict([PROD], th, a, b, y, ye, tq)
    assert np.max(np.abs(mu - mu_d)) <= 1e-8 * np.abs(mu_d).max()
    assert np.all(np.abs(va - va_d) <= 1e-7 * va_d + 1e-11)

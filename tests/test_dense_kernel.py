"""Pins for the dense integrated-GP reference (oracle.dense).

The closed-form double integral (second-antiderivative form) is checked
against the paper's equal-exposure celerite results (Appendix A: Eq.
delta-small for non-overlapping windows, the overlap formula, and the
simplified diagonal), with the SHO written as a celerite term
(a, b, c, d) = (sigma^2, sigma^2/(2 eta Q), omega0/(2Q), eta omega0), and
against adaptive 2-D quadrature for unequal and overlapping windows of SHO
and Matern-3/2 terms.
"""
import math

import numpy as np
import pytest
import scipy.integrate

from oracle import dense

SHO, M32 = 1, 2


def celerite_integrated(a, b, c, d, delta, lag):
    """Appendix A, equal exposure time delta, centres separated by lag."""
    C1 = a * c * c - a * d * d + 2 * b * c * d
    C2 = b * c * c - b * d * d - 2 * a * c * d
    den = delta ** 2 * (c * c + d * d) ** 2
    A = (2 * C1 * (math.cosh(c * delta) * math.cos(d * delta) - 1)
         - 2 * C2 * math.sinh(c * delta) * math.sin(d * delta)) / den
    B = (2 * C2 * (math.cosh(c * delta) * math.cos(d * delta) - 1)
         + 2 * C1 * math.sinh(c * delta) * math.sin(d * delta)) / den
    if lag == 0:
        return 2 * ((a * c + b * d) * (c * c + d * d) * delta - C1
                    + math.exp(-c * delta) * (C1 * math.cos(d * delta) + C2 * math.sin(d * delta))) / den
    base = A * math.exp(-c * lag) * math.cos(d * lag) + B * math.exp(-c * lag) * math.sin(d * lag)
    if delta <= lag:
        return base
    u = delta - lag
    return base + 2 * ((a * c + b * d) * (c * c + d * d) * u - C1 * math.sinh(c * u) * math.cos(d * u)
                       + C2 * math.cosh(c * u) * math.sin(d * u)) / (delta * (c * c + d * d)) ** 2


@pytest.mark.parametrize("q", [0.8, 3.0])
@pytest.mark.parametrize("delta", [0.1, 2.5])
@pytest.mark.parametrize("lag", [0.0, 0.05, 1.3, 7.0])
def test_equal_exposure_matches_appendix_a(q, delta, lag):
    sigma, w0 = 1.2, 1.7
    eta = math.sqrt(1 - 1 / (4 * q * q))
    a, b, c, d = sigma ** 2, sigma ** 2 / (2 * eta * q), w0 / (2 * q), eta * w0
    ref = celerite_integrated(a, b, c, d, delta, lag)
    t0 = 3.0
    ts = np.array([t0, t0 + lag])
    K = dense.integrated_cov([SHO], [sigma, w0, q, 0.1], ts, ts + delta)
    assert abs(K[0, 1] - ref) <= 1e-12 * max(abs(ref), sigma ** 2 * 1e-3)
    diag = celerite_integrated(a, b, c, d, delta, 0.0)
    assert abs(K[0, 0] - diag) <= 1e-12 * abs(diag)


def _quad2(kfun, a1, b1, a2, b2):
    # split at the kink |t - t'| = 0 when the windows overlap
    pts = sorted({a1, b1, a2, b2})
    tot = 0.0
    for i in range(len(pts) - 1):
        lo, hi = pts[i], pts[i + 1]
        if lo < max(a1, -1e300) or hi > b1:
            continue
        val, _ = scipy.integrate.dblquad(lambda tp, t: kfun(t - tp), lo, hi, a2, b2,
                                         epsabs=1e-13, epsrel=1e-12)
        tot += val
    return tot


@pytest.mark.parametrize("terms,theta", [([SHO], [0.9, 1.3, 2.0, 0.1]),
                                         ([M32], [1.1, 2.5, 0.1]),
                                         ([SHO, M32], [0.9, 1.3, 2.0, 0.5, 3.0, 0.1])])
@pytest.mark.parametrize("win", [((0.0, 1.0), (0.4, 2.9)),     # partial overlap, unequal
                                 ((0.0, 3.0), (1.0, 1.5)),     # nested
                                 ((0.0, 0.7), (2.2, 2.5)),     # separated
                                 ((0.0, 1.0), (1.0, 2.0))])    # touching
def test_unequal_overlapping_windows_match_quadrature(terms, theta, win):
    (a1, b1), (a2, b2) = win
    pars, _ = dense.split_theta(terms, theta)

    def k(x):
        return sum(dense.kernel(x, *p) for p in pars)

    ref = _quad2(k, a1, b1, a2, b2) / ((b1 - a1) * (b2 - a2))
    K = dense.integrated_cov(terms, theta, np.array([a1, a2]), np.array([b1, b2]))
    assert abs(K[0, 1] - ref) <= 1e-9 * abs(ref)
    assert abs(K[1, 0] - ref) <= 1e-9 * abs(ref)

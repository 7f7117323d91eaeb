"""Dense integrated-GP log-likelihood: the plain definition the filter must equal.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Definition (Section 2.1, Eq. full GP solution; Section 3.1): for exposure
windows [a_i, b_i] of lengths delta_i,

    K_ij = 1/(delta_i delta_j) * int_{a_i}^{b_i} int_{a_j}^{b_j} k(|t - t'|) dt dt'
    L    = -1/2 (y^T (K + R)^{-1} y + log det(K + R) + N log 2 pi),
    R    = diag(yerr^2 + s^2).

The double integral has a closed form for any lengths and any overlap: with G
the even second antiderivative of k(|x|) normalised by G(0) = G'(0) = 0,

    int_{a_i}^{b_i} int_{a_j}^{b_j} k = G(b_i - a_j) - G(a_i - a_j) - G(b_i - b_j) + G(a_i - b_j).

SHO with Q > 1/2 (Eq. sho_kernel): k(x) = Re(alpha e^{-beta x}) with
alpha = sigma^2 (1 - i/(2 eta Q)), beta = omega0/(2Q) - i eta omega0, hence
G(x) = Re(alpha (e^{-beta x} - 1 + beta x) / beta^2).
Matern-3/2 / critically damped SHO (Q = 1/2): k(x) = sigma^2 (1 + lam x) e^{-lam x},
G(x) = sigma^2 [2x/lam + (2/lam + x) e^{-lam x}/lam + e^{-lam x}/lam^2 - 3/lam^2].
Overdamped SHO (Q < 1/2; Eq. sho_kernel with eta = i sqrt(1/(4Q^2) - 1), so
cos and sin become cosh and sinh): with a = omega0/(2Q), b = omega0 sqrt(1/(4Q^2) - 1),
k(x) = sigma^2 e^{-a x} (cosh(b x) + (a/b) sinh(b x)), a sum of two real
exponentials c_pm e^{-lam_pm x}, c_pm = sigma^2 (1 pm a/b)/2, lam_pm = a -+ b,
each with G = c (e^{-lam x} - 1 + lam x) / lam^2.
"""
from __future__ import annotations

import math
import numpy as np
import scipy.integrate
import scipy.linalg

SHO = 1
MATERN32 = 2
SHO_PRODUCT = 3


def split_theta(terms, theta):
    """Per-term (sigma, omega0, Q) and white-noise sd from natural parameters;
    a product of two SHOs gives (sigma, omega_a, Q_a, omega_b, Q_b)."""
    out = []
    j = 0
    for k in terms:
        if k == SHO:
            out.append((theta[j], theta[j + 1], theta[j + 2]))
            j += 3
        elif k == SHO_PRODUCT:
            out.append(tuple(theta[j:j + 5]))
            j += 5
        else:
            out.append((theta[j], math.sqrt(3.0) / theta[j + 1], 0.5))
            j += 2
    return out, theta[j]


def term_kernel(x, p):
    """k(|x|) of one term: an SHO / Matern-3/2 (sigma, omega0, Q), or a product
    of two SHOs sigma^2 k_a k_b with unit-variance factors (Appendix C.2)."""
    if len(p) == 3:
        return kernel(x, *p)
    sig, wa, qa, wb, qb = p
    return sig ** 2 * kernel(x, 1.0, wa, qa) * kernel(x, 1.0, wb, qb)


def _quad_window(kfun, t, a, b):
    """int_a^b k(t - s) ds by adaptive quadrature (split at s = t)."""
    pts = [t] if a < t < b else None
    v, _ = scipy.integrate.quad(lambda u: kfun(t - u), a, b, points=pts, epsabs=1e-14,
                                epsrel=1e-12, limit=200)
    return v


def _quad_pair(kfun, a1, b1, a2, b2):
    """int_{a1}^{b1} int_{a2}^{b2} k(t - t') by nested quadrature."""
    return scipy.integrate.quad(lambda t: _quad_window(kfun, t, a2, b2), a1, b1,
                                points=[p for p in (a2, b2) if a1 < p < b1] or None,
                                epsabs=1e-13, epsrel=1e-11, limit=200)[0]


def overdamped_modes(sigma, w0, q, dtype=np.float64):
    """The two real exponentials (c, lam) of the overdamped SHO kernel; the slow
    rate a - b is formed as omega0^2 / (a + b) (no cancellation)."""
    sigma, w0, q = dtype(sigma), dtype(w0), dtype(q)
    a = w0 / (2 * q)
    b = w0 * np.sqrt(1 / (4 * q * q) - 1)
    return [(sigma ** 2 * (1 + a / b) / 2, w0 * w0 / (a + b)),
            (sigma ** 2 * (1 - a / b) / 2, a + b)]


def kernel(x, sigma, w0, q):
    """Stationary SHO kernel k(|x|) (Eq. sho_kernel), any Q > 0."""
    x = np.abs(x)
    if q == 0.5:
        return sigma ** 2 * (1 + w0 * x) * np.exp(-w0 * x)
    if q < 0.5:
        return sum(c * np.exp(-lam * x) for c, lam in overdamped_modes(sigma, w0, q))
    eta = math.sqrt(1 - 1 / (4 * q * q))
    return sigma ** 2 * np.exp(-w0 * x / (2 * q)) * (
        np.cos(eta * w0 * x) + np.sin(eta * w0 * x) / (2 * eta * q))


def G(x, sigma, w0, q):
    """Even second antiderivative of k(|x|) with G(0) = G'(0) = 0.

    Evaluated in extended precision: the four-term combination below
    cancels to O(delta^2) for short exposures."""
    LD = np.longdouble
    x = np.abs(np.asarray(x, LD))
    sigma, w0, q = LD(sigma), LD(w0), LD(q)
    if q == 0.5:
        lam = w0
        e = np.exp(-lam * x)
        return sigma ** 2 * (2 * x / lam + (2 / lam + x) * e / lam + e / lam ** 2 - 3 / lam ** 2)
    if q < 0.5:
        return sum(c * (np.exp(-lam * x) - 1 + lam * x) / lam ** 2
                   for c, lam in overdamped_modes(sigma, w0, q, LD))
    eta = np.sqrt(1 - 1 / (4 * q * q))
    alpha = sigma ** 2 * (1 - np.clongdouble(1j) / (2 * eta * q))
    beta = w0 / (2 * q) - np.clongdouble(1j) * eta * w0
    return np.real(alpha * (np.exp(-beta * x) - 1 + beta * x) / beta ** 2)


def integrated_cov(terms, theta, t_start, t_end):
    """K_ij of exposure-averaged values for a sum of SHO / Matern-3/2 terms.

    A measurement with t_start == t_end is instantaneous (the limit delta -> 0
    of the exposure average, Section 3.2: z / delta -> f): its covariance with
    another instantaneous one is k(|t_i - t_j|), with an exposure [a, b] of
    length delta it is (F1(t - a) - F1(t - b)) / delta."""
    a = np.asarray(t_start, np.longdouble)
    b = np.asarray(t_end, np.longdouble)
    d = b - a
    inst = d == 0
    pars_all, _ = split_theta(terms, theta)
    pars = [p for p in pars_all if len(p) == 3]
    prods = [p for p in pars_all if len(p) == 5]
    n = len(a)
    K = np.zeros((n, n), np.longdouble)
    for sigma, w0, q in pars:
        K += (G(b[:, None] - a[None, :], sigma, w0, q) - G(a[:, None] - a[None, :], sigma, w0, q)
              - G(b[:, None] - b[None, :], sigma, w0, q) + G(a[:, None] - b[None, :], sigma, w0, q))
    dd = np.where(inst, 1, d)
    K = (K / (dd[:, None] * dd[None, :])).astype(np.float64)
    if inst.any():
        t = np.asarray(t_start, np.float64)
        ta, tb, dl = t, np.asarray(t_end, np.float64), np.where(inst, 1.0, np.asarray(d, np.float64))
        ki = np.nonzero(inst)[0]
        cross = np.zeros((len(ki), n))
        kk = np.zeros((len(ki), len(ki)))
        for sigma, w0, q in pars:
            cross += (F1(t[ki, None] - ta[None, :], sigma, w0, q) -
                      F1(t[ki, None] - tb[None, :], sigma, w0, q)) / dl[None, :]
            kk += kernel(t[ki, None] - t[None, ki], sigma, w0, q)
        K[ki, :] = cross
        K[:, ki] = cross.T
        K[np.ix_(ki, ki)] = kk
    if prods:
        # products (no closed form here): quadrature of the kernel, for small N
        ta, tb = np.asarray(t_start, np.float64), np.asarray(t_end, np.float64)
        kfun = lambda x: sum(term_kernel(x, p) for p in prods)
        for i in range(n):
            for j in range(i, n):
                if inst[i] and inst[j]:
                    v = kfun(ta[i] - ta[j])
                elif inst[i]:
                    v = _quad_window(kfun, ta[i], ta[j], tb[j]) / (tb[j] - ta[j])
                elif inst[j]:
                    v = _quad_window(kfun, ta[j], ta[i], tb[i]) / (tb[i] - ta[i])
                else:
                    v = _quad_pair(kfun, ta[i], tb[i], ta[j], tb[j]) / (
                        (tb[i] - ta[i]) * (tb[j] - ta[j]))
                K[i, j] += v
                if j != i:
                    K[j, i] += v
    return K


def instantaneous_cov(terms, theta, t):
    t = np.asarray(t, np.float64)
    pars, _ = split_theta(terms, theta)
    K = np.zeros((len(t), len(t)))
    for p in pars:
        K += term_kernel(t[:, None] - t[None, :], p)
    return K


def gaussian_loglik(K, y, noise_var):
    """-1/2 (y^T C^{-1} y + log det C + N log 2 pi), C = K + diag(noise_var)."""
    C = K + np.diag(noise_var)
    c, low = scipy.linalg.cho_factor(C, lower=True)
    alpha = scipy.linalg.cho_solve((c, low), y)
    return -0.5 * (y @ alpha + 2 * np.sum(np.log(np.diag(c))) + len(y) * math.log(2 * math.pi))


def loglik(terms, theta, t_start, t_end, y, yerr):
    """Dense integrated-GP log-likelihood (N <= ~2000)."""
    _, s = split_theta(terms, theta)
    K = integrated_cov(terms, theta, t_start, t_end)
    y = np.asarray(y, np.float64)
    return gaussian_loglik(K, y, np.asarray(yerr, np.float64) ** 2 + s * s)


def loglik_instantaneous(terms, theta, t, y, yerr):
    """Dense log-likelihood of instantaneous measurements at times t."""
    _, s = split_theta(terms, theta)
    K = instantaneous_cov(terms, theta, t)
    return gaussian_loglik(K, np.asarray(y, np.float64), np.asarray(yerr, np.float64) ** 2 + s * s)


def posterior(terms, theta, t_start, t_end, y, yerr):
    """Conditioned mean and variance of every exposure average given all the
    data: K (K + R)^-1 y and diag(K - K (K + R)^-1 K), with K the integrated
    kernel of the exposure averages and R = diag(yerr^2 + s^2) (the full GP
    solution of Section 2 with the integrated kernel of Section 3.1)."""
    _, s = split_theta(terms, theta)
    K = integrated_cov(terms, theta, t_start, t_end)
    A = K + np.diag(np.asarray(yerr, np.float64) ** 2 + s * s)
    y = np.asarray(y, np.float64)
    return K @ np.linalg.solve(A, y), np.diag(K - K @ np.linalg.solve(A, K))


def F1(x, sigma, w0, q):
    """Odd first antiderivative of k(|x|), F1(0) = 0 (the derivative of G)."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    if q == 0.5:
        lam = w0
        v = sigma ** 2 * (2 / lam - np.exp(-lam * a) * (2 / lam + a))
    elif q < 0.5:
        v = sum(c * -np.expm1(-lam * a) / lam for c, lam in overdamped_modes(sigma, w0, q))
    else:
        eta = math.sqrt(1 - 1 / (4 * q * q))
        alpha = sigma ** 2 * (1 - 1j / (2 * eta * q))
        beta = w0 / (2 * q) - 1j * eta * w0
        v = np.real(alpha * (1 - np.exp(-beta * a)) / beta)
    return np.sign(x) * v


def predict(terms, theta, t_start, t_end, y, yerr, t_star):
    """Mean and variance of the latent f(t*) given exposure-averaged data:
    k*^T (K + R)^-1 y and k(0) - k*^T (K + R)^-1 k*, with
    k*_n = cov(f(t*), average over exposure n) = (F1(t* - ts_n) - F1(t* - te_n)) / delta_n."""
    pars, s = split_theta(terms, theta)
    ts_, te_ = np.asarray(t_start, np.float64), np.asarray(t_end, np.float64)
    d = te_ - ts_
    K = integrated_cov(terms, theta, ts_, te_)
    A = K + np.diag(np.asarray(yerr, np.float64) ** 2 + s * s)
    t_star = np.asarray(t_star, np.float64)
    ks = np.zeros((len(t_star), len(ts_)))
    k0 = 0.0
    inst = d == 0
    dl = np.where(inst, 1.0, d)
    for p in pars:
        k0 += p[0] ** 2
        if len(p) == 5:  # product: quadrature over each window (small cases)
            for i, tq in enumerate(t_star):
                for n in range(len(ts_)):
                    ks[i, n] += (term_kernel(tq - ts_[n], p) if inst[n] else
                                 _quad_window(lambda x: term_kernel(x, p), tq, ts_[n], te_[n]) / d[n])
            continue
        sig, w0, q = p
        ks += np.where(inst[None, :], kernel(t_star[:, None] - ts_[None, :], sig, w0, q),
                       (F1(t_star[:, None] - ts_[None, :], sig, w0, q) -
                        F1(t_star[:, None] - te_[None, :], sig, w0, q)) / dl[None, :])
    sol = np.linalg.solve(A, np.c_[np.asarray(y, np.float64), ks.T])
    mean = ks @ sol[:, 0]
    var = k0 - np.einsum("ij,ji->i", ks, sol[:, 1:])
    return mean, var

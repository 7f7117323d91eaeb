"""Pins for the oracle's discretisation (Van Loan + exact doubling).

Each check fixes Phi~(dt), Q~(dt) by something other than the oracle itself:
  * the paper's printed SHO closed forms (Appendix B: Eqs. sho_phi, sho_Q,
    sho_phibar, analytic_Qaug12, analytic_Qaug22), evaluated in 40-digit
    arithmetic with mpmath so that their own cancellation does not matter;
  * adaptive quadrature of the defining integrals (Eq. phiaug for
    Phibar = int Phi, Eq. Q_aug for Q~) with scipy's expm as the integrand;
  * the Q = 1/2 transition of Eq. sho_phi and the identity Q = P_inf - A P_inf A^T
    (Eq. Q);
  * semigroup identities and stationarity for long steps;
  * the block layout of several integral states (Section 3.2.3) and of sums
    of terms (Appendix C.1).
"""
import math

import mpmath as mp
import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle

SHO, M32 = 1, 2
mp.mp.dps = 40


def printed_sho_blocks(sigma, w0, q, dt):
    """Appendix B closed forms for Q > 1/2, transcribed from the paper."""
    sigma, w0, q, dt = (mp.mpf(v) for v in (sigma, w0, q, dt))
    eta = mp.sqrt(1 - 1 / (4 * q * q))
    tau = eta * w0 * dt
    A = 1 / (2 * eta * q)
    e1 = mp.e ** (-w0 * dt / (2 * q))
    e2 = mp.e ** (-w0 * dt / q)
    Phi = e1 * mp.matrix([[mp.cos(tau) + A * mp.sin(tau), mp.sin(tau) / (eta * w0)],
                          [-w0 / eta * mp.sin(tau), mp.cos(tau) - A * mp.sin(tau)]])
    s2 = mp.sin(tau) ** 2
    qaa = mp.e ** (w0 * dt / q) - 1 - A * mp.sin(2 * tau) - s2 / (2 * eta ** 2 * q ** 2)
    qab = w0 / (eta ** 2 * q) * s2
    qbb = w0 ** 2 * (mp.e ** (w0 * dt / q) - 1 + A * mp.sin(2 * tau) - s2 / (2 * eta ** 2 * q ** 2))
    Qk = sigma ** 2 * e2 * mp.matrix([[qaa, qab], [qab, qbb]])
    # Eq. sho_phibar, first row only
    a = -w0 / (2 * q)
    b = eta * w0
    B = 1 / (eta * w0)

    def prim(t):
        tt = b * t
        Is = a * mp.sin(tt) - b * mp.cos(tt)
        Ic = a * mp.cos(tt) + b * mp.sin(tt)
        f = mp.e ** (a * t) / (a * a + b * b)
        return f * (Ic + A * Is), f * (B * Is)

    p1, p0 = prim(dt), prim(0)
    phibar = [p1[0] - p0[0], p1[1] - p0[1]]
    q12 = sigma ** 2 * mp.matrix([
        [1 / (q * w0) * (e1 * (mp.cos(tau) + A * mp.sin(tau)) - 1) ** 2],
        [A * e1 * (4 * mp.sin(tau) - e1 * mp.sin(2 * tau)) - 2 * A ** 2 * e2 * s2 + e2 - 1]])
    q22 = sigma ** 2 / (4 * q ** 2 * w0 ** 2) * (
        8 * q * w0 * dt + 4 * q ** 2 - 12 + A ** 2 * e2 * (mp.cos(2 * tau) - 16 * q ** 4)
        + 16 * e1 * (mp.cos(tau) + (1 - 2 * q ** 2) * A * mp.sin(tau))
        + e2 * ((1 - 3 * A ** 2) / A * mp.sin(2 * tau) - 3 * mp.cos(2 * tau)))
    Phit = np.zeros((3, 3))
    Qt = np.zeros((3, 3))
    for i in range(2):
        for j in range(2):
            Phit[i, j] = float(Phi[i, j])
            Qt[i, j] = float(Qk[i, j])
        Phit[2, i] = float(phibar[i])
        Qt[i, 2] = Qt[2, i] = float(q12[i])
    Phit[2, 2] = 1.0
    Qt[2, 2] = float(q22)
    return Phit, Qt


def close(a, b, rtol=5e-11, ntol=1e-14):
    """|a - b| <= rtol |b| + ntol max|b| elementwise: relative for entries of
    the matrix's own scale, normwise (a few ulps of the largest entry) for
    entries that are small differences of large ones."""
    return bool(np.all(np.abs(a - b) <= rtol * np.abs(b) + ntol * np.max(np.abs(b))))


@pytest.mark.parametrize("q", [0.8, 3.0, 10.0])
@pytest.mark.parametrize("w0", [2 * math.pi / 10, 3.0])
@pytest.mark.parametrize("dt", [1e-3, 0.05, 0.7, 4.0, 40.0])
def test_van_loan_matches_printed_closed_forms(oracle_lib, q, w0, dt):
    theta = [1.3, w0, q, 0.1]
    Phi, Q, _ = oracle.discretize([SHO], 0, 1, theta, dt)
    Phic, Qc = printed_sho_blocks(1.3, w0, q, dt)
    # entries that are exactly zero (the z column of Phi~) must match exactly
    assert Phi[0, 2] == 0 and Phi[1, 2] == 0 and Phi[2, 2] == 1.0
    assert close(Phi, Phic)
    assert close(Q, Qc)


def _phi_aug(theta_row, dt, terms=(SHO,), layout=0, n_slots=1):
    Phi, Q, P0 = oracle.discretize(list(terms), layout, n_slots, theta_row, dt)
    return Phi, Q, P0


def _F_and_LQL(sigma, w0, q):
    F = np.array([[0.0, 1.0, 0.0], [-w0 * w0, -w0 / q, 0.0], [1.0, 0.0, 0.0]])
    LQL = np.zeros((3, 3))
    LQL[1, 1] = 2 * w0 ** 3 * sigma ** 2 / q
    return F, LQL


@pytest.mark.parametrize("q", [0.5, 0.7, 3.0])
@pytest.mark.parametrize("dt", [0.02, 0.9, 6.0])
def test_van_loan_matches_quadrature(oracle_lib, q, dt):
    sigma, w0 = 0.8, 1.1
    F, LQL = _F_and_LQL(sigma, w0, q)
    theta = [sigma, w0, q, 0.1] if q != 0.5 else [sigma, math.sqrt(3) / w0, 0.1]
    terms = [SHO] if q != 0.5 else [M32]
    Phi, Q, _ = _phi_aug(theta, dt, terms)
    np.testing.assert_allclose(Phi, scipy.linalg.expm(F * dt), rtol=1e-12, atol=1e-15)
    # Phibar = int_0^dt Phi(s) ds (Eq. phiaug); z row of Phi~
    F2 = F[:2, :2]
    for j in range(2):
        val, _ = scipy.integrate.quad(lambda s: scipy.linalg.expm(F2 * s)[0, j], 0, dt,
                                      epsabs=0, epsrel=1e-12, limit=200)
        assert abs(Phi[2, j] - val) <= 1e-11 * max(abs(val), 1e-12)
    # Q~ = int_0^dt Phi~(s) L~ Qc L~^T Phi~(s)^T ds (Eq. Q_aug)
    for i in range(3):
        for j in range(i, 3):
            def integrand(s, i=i, j=j):
                E = scipy.linalg.expm(F * s)
                return (E @ LQL @ E.T)[i, j]
            val, _ = scipy.integrate.quad(integrand, 0, dt, epsabs=0, epsrel=1e-12, limit=200)
            assert abs(Q[i, j] - val) <= 1e-10 * max(abs(val), 1e-14 * abs(Q).max()), (i, j)


@pytest.mark.parametrize("dt", [0.01, 0.5, 3.0])
def test_critical_damping_transition_and_lyapunov_identity(oracle_lib, dt):
    ell, sigma = 4.0, 0.7
    w0 = math.sqrt(3) / ell
    Phi, Q, P0 = _phi_aug([sigma, ell, 0.1], dt, [M32])
    e = math.exp(-w0 * dt)
    printed = e * np.array([[1 + w0 * dt, dt], [-w0 * w0 * dt, 1 - w0 * dt]])
    np.testing.assert_allclose(Phi[:2, :2], printed, rtol=1e-13, atol=1e-16)
    Pinf = P0[:2, :2]
    np.testing.assert_allclose(Pinf, sigma ** 2 * np.diag([1, w0 * w0]), rtol=1e-15)
    lyap = Pinf - printed @ Pinf @ printed.T
    np.testing.assert_allclose(Q[:2, :2], lyap, rtol=1e-9, atol=1e-13 * sigma ** 2)


def test_semigroup_and_stationarity(oracle_lib):
    theta = [1.0, 2 * math.pi / 10, 3.0, 0.5, 5.0, 0.1]
    terms = [SHO, M32]
    a, b = 0.37, 1.91
    Pa, Qa, _ = _phi_aug(theta, a, terms)
    Pb, Qb, _ = _phi_aug(theta, b, terms)
    Pab, Qab, P0 = _phi_aug(theta, a + b, terms)
    np.testing.assert_allclose(Pab, Pb @ Pa, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Qab, Pb @ Qa @ Pb.T + Qb, rtol=1e-11, atol=1e-13)
    # a very long step forgets the state: Phi -> 0, Q_x -> P_inf
    Pl, Ql, P0 = _phi_aug(theta, 5000.0, terms)
    np.testing.assert_allclose(Pl[:4, :4], 0, atol=1e-12)
    np.testing.assert_allclose(Ql[:4, :4], P0[:4, :4], rtol=1e-10, atol=1e-12)
    assert Ql[4, 4] > 0


def test_multi_slot_and_sum_block_structure(oracle_lib):
    """Section 3.2.3: every z row of Phi~ carries Phibar_x, every z column of
    Q~ carries Q~12 and the whole z block is Q~22.  Appendix C.1: terms are
    independent (block-diagonal x part) and z integrates the sum H x."""
    theta = [1.0, 0.9, 2.0, 0.5, 3.0, 0.1]
    dt = 0.8
    P1, Q1, _ = _phi_aug(theta, dt, [SHO, M32], 0, 1)
    P3, Q3, _ = _phi_aug(theta, dt, [SHO, M32], 0, 3)
    for j in range(3):
        np.testing.assert_allclose(P3[4 + j, :4], P1[4, :4], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(Q3[:4, 4 + j], Q1[:4, 4], rtol=1e-12, atol=1e-15)
        for k in range(3):
            assert abs(Q3[4 + j, 4 + k] - Q1[4, 4]) <= 1e-12 * Q1[4, 4]
    # single-term models reproduce the sum's diagonal blocks
    Ps, Qs, _ = _phi_aug([1.0, 0.9, 2.0, 0.1], dt, [SHO])
    Pm, Qm, _ = _phi_aug([0.5, 3.0, 0.1], dt, [M32])
    np.testing.assert_allclose(P1[:2, :2], Ps[:2, :2], rtol=1e-13)
    np.testing.assert_allclose(P1[2:4, 2:4], Pm[:2, :2], rtol=1e-13)
    np.testing.assert_allclose(P1[4, :2], Ps[2, :2], rtol=1e-13)
    np.testing.assert_allclose(P1[4, 2:4], Pm[2, :2], rtol=1e-13)
    np.testing.assert_allclose(Q1[4, 4], Qs[2, 2] + Qm[2, 2], rtol=1e-12)
    np.testing.assert_allclose(Q1[:2, 2:4], 0, atol=1e-15)
    # layout 1: one z per term, each integrating only its own term
    P1l, Q1l, _ = _phi_aug(theta, dt, [SHO, M32], 1, 1)
    np.testing.assert_allclose(P1l[4, :2], Ps[2, :2], rtol=1e-13)
    np.testing.assert_allclose(P1l[4, 2:4], 0, atol=1e-15)
    np.testing.assert_allclose(Q1l[5, 5], Qm[2, 2], rtol=1e-12)
    assert abs(Q1l[4, 5]) <= 1e-15


@pytest.mark.parametrize("q", [0.55, 3.0, 10.0])
@pytest.mark.parametrize("dt", [0.05, 0.7, 4.0, 40.0, 400.0])
@pytest.mark.parametrize("layout,n_slots", [(0, 1), (0, 3), (1, 2)])
def test_closed_form_timing_mode_matches_van_loan(oracle_lib, q, dt, layout, n_slots):
    # the timing mode's per-term closed forms (Appendix B), assembled for a sum
    # of two SHO terms and several integral states, against Van Loan of the
    # whole augmented model
    theta = [1.3, 0.9, q, 0.6, 2.5, 1.7, 0.1]
    Pv, Qv, _ = oracle.discretize([SHO, SHO], layout, n_slots, theta, dt)
    Pc, Qc, _ = oracle.discretize([SHO, SHO], layout, n_slots, theta, dt, closed_form=True)
    assert close(Pc, Pv, rtol=1e-9, ntol=1e-12)
    assert close(Qc, Qv, rtol=1e-9, ntol=1e-12)


@pytest.mark.parametrize("dt", [0.05, 0.7, 4.0, 40.0, 400.0])
@pytest.mark.parametrize("layout,n_slots", [(0, 1), (0, 3), (1, 2)])
def test_closed_form_timing_mode_critical_damping(oracle_lib, dt, layout, n_slots):
    # Matern-3/2 (and an SHO at Q = 1/2 exactly): Phi of Eq. sho_phi, Q from
    # Eq. Q and the integrated blocks worked out from their defining integrals
    for terms, theta in (([SHO, M32], [1.0, 2.0, 3.0, 0.5, 4.0, 0.1]),
                         ([SHO, SHO], [1.0, 0.9, 0.5, 0.6, 2.5, 1.7, 0.1])):
        Pv, Qv, _ = oracle.discretize(terms, layout, n_slots, theta, dt)
        Pc, Qc, _ = oracle.discretize(terms, layout, n_slots, theta, dt, closed_form=True)
        assert close(Pc, Pv, rtol=1e-9, ntol=1e-12)
        assert close(Qc, Qv, rtol=1e-9, ntol=1e-12)


def test_closed_form_timing_mode_falls_back():
    # an overdamped SHO (Q < 1/2) has no closed forms printed for Q~: Van Loan
    theta = [1.0, 2.0, 0.3, 0.5, 4.0, 0.1]
    Pv, Qv, _ = oracle.discretize([SHO, M32], 0, 1, theta, 0.3)
    Pc, Qc, _ = oracle.discretize([SHO, M32], 0, 1, theta, 0.3, closed_form=True)
    assert np.array_equal(Pc, Pv) and np.array_equal(Qc, Qv)


def test_closed_form_timing_mode_loglik_and_gradient(oracle_lib):
    # the filter in the timing mode gives the Van Loan log-likelihood and
    # complex-step gradient to within 1e-8 per measurement (c1, c2 and c4
    # recipes; the closed forms lose digits to cancellation at short steps)
    import synth
    for wl in (synth.c1(), synth.c4(n_series=2, scale=0.1), synth.c2(n_series=2, scale=0.05)):
        for i in range(wl.n_series):
            ts, te, y, ye, _ = wl.series(i)
            k = min(len(ts), 800)
            a, ga = oracle.loglik(wl.terms, wl.layout, ts[:k], te[:k], y[:k], ye[:k],
                                  wl.theta[i], grad=True)
            b, gb = oracle.loglik(wl.terms, wl.layout, ts[:k], te[:k], y[:k], ye[:k],
                                  wl.theta[i], grad=True, closed_form=True)
            assert abs(a - b) <= 1e-8 * k
            assert np.all(np.abs(ga - gb) <= 1e-6 * np.abs(ga) + 1e-8 * k)

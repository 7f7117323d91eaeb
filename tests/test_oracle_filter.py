"""Pins for the oracle's sequential integrated Kalman filter.

* Equivalence with the dense integrated GP (Section 4: the integrated SSM and
  the fully integrated GP give the same likelihood to ~1e-14): single
  instrument with and without dead time, sums of terms, two overlapping
  instruments, three concurrently open exposures, unlabelled data (greedy
  slots), and one-integral-state-per-term layout.
* Invariants: covariance symmetric and PSD along the trajectory, S > 0,
  invariance to a common time shift, to instrument relabelling, and the
  end-before-start tie rule (reading G1) being the one the dense GP agrees with.
* The instantaneous limit: as every exposure shrinks around a fixed midpoint
  the likelihood tends to the dense instantaneous GP likelihood (Section 3.2:
  z / delta -> x), with an O(delta^2) gap.
* Gradients: complex-step derivatives vs central finite differences.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import dense

SHO, M32 = 1, 2
TOL = 1e-9


def _check_dense(terms, layout, ts, te, y, ye, theta, inst=None):
    lk = oracle.loglik(terms, layout, ts, te, y, ye, theta, instrument=inst)
    ld = dense.loglik(terms, theta, ts, te, y, ye)
    assert abs(lk - ld) <= TOL * abs(ld), (lk, ld)
    return lk


@pytest.mark.parametrize("seed,n", [(11, 300), (12, 57)])
def test_single_sho_matches_dense(oracle_lib, seed, n):
    wl = synth.small_single(seed, n, [SHO], [1.0, 2 * math.pi / 10, 3.0, 0.1])
    ts, te, y, ye, _ = wl.series(0)
    _check_dense([SHO], 0, ts, te, y, ye, wl.theta[0])


def test_sum_of_terms_and_layouts_match_dense(oracle_lib):
    th = [1.0, 2 * math.pi / 10, 3.0, 0.5, 5.0, 0.1]
    wl = synth.small_single(13, 250, [SHO, M32], th)
    ts, te, y, ye, _ = wl.series(0)
    l0 = _check_dense([SHO, M32], 0, ts, te, y, ye, wl.theta[0])
    l1 = _check_dense([SHO, M32], 1, ts, te, y, ye, wl.theta[0])
    assert abs(l0 - l1) <= 1e-12 * abs(l0)
    th2 = [1.0, 2 * math.pi / 10, 3.0, 0.5, math.pi, 1.0, 0.1]
    wl = synth.small_single(14, 200, [SHO, SHO], th2)
    ts, te, y, ye, _ = wl.series(0)
    a = _check_dense([SHO, SHO], 0, ts, te, y, ye, wl.theta[0])
    b = _check_dense([SHO, SHO], 1, ts, te, y, ye, wl.theta[0])
    assert abs(a - b) <= 1e-12 * abs(a)


def test_no_dead_time_single_instrument(oracle_lib):
    """Section 4, Fig. 2 shape: 180 s exposures back to back, SHO with a
    ~300 s period, sigma_y = 0.3."""
    rng = np.random.default_rng(21)
    n = 120
    ts = np.arange(n) * 180.0
    te = ts + 180.0
    y = rng.normal(0, 1, n).astype(np.float32)
    ye = np.zeros(n, np.float32)
    theta = [1.0, 2 * math.pi / 300, 3.0, 0.3]
    lk = _check_dense([SHO], 0, ts, te, y, ye, theta)
    # the other tie order (start before end at equal times) is wrong
    ev = oracle.events(ts, te, y, ye)
    bad = dict(ev)
    order = np.lexsort((ev["meas"], ev["kind"], ev["t"]))  # starts first at ties
    for k in ("t", "kind", "slot", "meas", "y", "r0", "invd"):
        bad[k] = ev[k][order]
    lb = oracle.loglik_events([SHO], 0, bad, theta)["loglik"]
    assert abs(lb - lk) > 1e-3 * abs(lk)


def test_two_overlapping_instruments(oracle_lib):
    """Section 4, Fig. 3 shape: 55 s exposures and 180 +- 30 s exposures."""
    wl = synth.two_instrument_overlap(3, 90, 30)
    ts, te, y, ye, inst = wl.series(0)
    l_lab = _check_dense([SHO], 0, ts, te, y, ye, wl.theta[0], inst)
    l_greedy = oracle.loglik([SHO], 0, ts, te, y, ye, wl.theta[0])
    assert abs(l_lab - l_greedy) <= 1e-12 * abs(l_lab)
    # relabelling instruments permutes the integral states only
    l_swap = oracle.loglik([SHO], 0, ts, te, y, ye, wl.theta[0], instrument=1 - inst)
    assert abs(l_lab - l_swap) <= 1e-12 * abs(l_lab)
    # extra, never-used slots change nothing
    l_extra = oracle.loglik([SHO], 0, ts, te, y, ye, wl.theta[0], instrument=inst, n_slots=4)
    assert abs(l_lab - l_extra) <= 1e-12 * abs(l_lab)


def test_three_concurrently_open(oracle_lib):
    rng = np.random.default_rng(5)
    ts, te, slot = synth.capped_overlap_exposures(rng, 240, 0.5, 0.5, 3.0, cap=3)
    y = rng.normal(0, 1, len(ts)).astype(np.float32)
    ye = np.full(len(ts), 0.05, np.float32)
    theta = [1.0, 2 * math.pi / 10, 3.0, 0.1]
    lk = _check_dense([SHO], 0, ts, te, y, ye, theta, slot)
    ev = oracle.events(ts, te, y, ye, slot)
    assert ev["n_slots"] == 3


def test_self_overlap_rejected(oracle_lib):
    with pytest.raises(oracle.SelfOverlapError):
        oracle.events([0.0, 0.5], [1.0, 1.5], [0, 0], [0, 0], instrument=[0, 0])


def test_invariants_along_trajectory(oracle_lib):
    wl = synth.two_instrument_overlap(4, 60, 25)
    ts, te, y, ye, inst = wl.series(0)
    ev = oracle.events(ts, te, y, ye, inst)
    r = oracle.loglik_events([SHO], 0, ev, wl.theta[0], dump=True)
    P = r["P"]
    assert np.all(r["S"] > 0)
    asym = np.max(np.abs(P - np.transpose(P, (0, 2, 1))))
    assert asym == 0.0
    for Pk in P:
        lam = np.linalg.eigvalsh(Pk)
        assert lam.min() >= -1e-12 * max(lam.max(), 1.0)
    # a common time shift changes nothing (stationarity)
    l0 = r["loglik"]
    l1 = oracle.loglik([SHO], 0, ts + 12345.0, te + 12345.0, y, ye, wl.theta[0], instrument=inst)
    assert abs(l0 - l1) <= 1e-9 * abs(l0)


def test_instantaneous_limit(oracle_lib):
    rng = np.random.default_rng(31)
    n = 150
    tm = np.cumsum(rng.exponential(1.0, n))
    y = rng.normal(0, 1, n)
    ye = np.zeros(n)
    theta = [1.0, 2 * math.pi / 10, 3.0, 0.1]
    linst = dense.loglik_instantaneous([SHO], theta, tm, y, ye)
    gaps = []
    for d in [0.04, 0.02, 0.01]:
        li = oracle.loglik([SHO], 0, tm - d / 2, tm + d / 2, y, ye, theta)
        gaps.append(li - linst)
    r1, r2 = gaps[0] / gaps[1], gaps[1] / gaps[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, gaps
    assert abs(gaps[-1]) < 1e-3 * abs(linst)


@pytest.mark.parametrize("terms,layout,theta", [
    ([SHO], 0, [1.0, 2 * math.pi / 10, 3.0, 0.1]),
    ([SHO, M32], 0, [1.0, 0.8, 2.0, 0.5, 4.0, 0.15]),
    ([SHO, SHO], 1, [1.0, 0.7, 3.0, 0.5, 3.0, 1.2, 0.1])])
def test_complex_step_gradient_matches_central_differences(oracle_lib, terms, layout, theta):
    wl = synth.small_single(41, 120, terms, theta)
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
        # Richardson-extrapolated central difference: truncation O(h^4)
        fd = (4 * central(i, h / 2) - central(i, h)) / 3
        assert abs(fd - g[i]) <= 1e-7 * max(abs(g[i]), 1e-2 * abs(l0)), (i, fd, g[i])

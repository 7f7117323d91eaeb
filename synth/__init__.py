"""Seeded synthetic workloads for integrated, possibly overlapping exposures.

This module only draws inputs: exposure windows, instrument labels, observed
exposure averages and hyperparameter vectors.  It holds none of the
likelihood method's arithmetic (no state-space model, discretisation or
filtering); both the FP64 oracle and the CUDA path consume what it returns.

Observed values.  The latent signal is a random-Fourier-feature draw of the
kernel (frequencies sampled from each term's power spectrum, Eq. sho_psd),
averaged analytically over each exposure window, plus white noise of standard
deviation ``s``.  The log-likelihood is defined for any ``y``, so the draw
only has to have the right magnitude and smoothness; it is an approximate
sample of the model, not an exact one.

Workload shapes (Section 4 of the paper measures on synthetic SHO draws):

* ``c1`` one series, N = 1000, one SHO term, start gaps ~ Exp(1), exposure
  lengths ~ U[0.05, 0.5] clipped to the gap to the next start.
* ``c2`` 4096 series, N ~ log-uniform[500, 20000], SHO + Matern-3/2, every
  kernel parameter log-uniform over a factor 10 around its centre.
* ``c3`` one series, N = 2^22, start gaps ~ Exp(0.5), lengths ~ U[0.5, 3],
  at most 3 exposures open at once (a start that would open a 4th is moved to
  the earliest open end and takes that exposure's slot).
* ``c4`` 1024 series, N ~ U{2000..20000}, two SHO terms, parameters
  log-uniform over a factor 10, Q truncated at >= 0.55.
* ``c5`` one series of 1e6 measurements from 3 instruments with exposure
  lengths 0.1 / 1 / 5 (start gaps delta_i + Exp(delta_i)), shared by 256
  hyperparameter vectors drawn log-normal(ln centre, 0.5).

Every generator takes a ``scale`` (fraction of the full size) so that the
same recipe yields the small cases the oracle finishes in seconds.
"""
from __future__ import annotations

import dataclasses
import heapq
import math

import numpy as np

TWO_PI = 2.0 * math.pi

# kernel term kinds (match the C ABI enum values)
SHO = 1
MATERN32 = 2
SHO_PRODUCT = 3


@dataclasses.dataclass
class Workload:
    """A batch of series sharing one kernel structure.

    Arrays are concatenated over series; ``offsets`` (int64, n_series+1)
    delimits each series.  ``theta`` is [n_sets, n_params] float64 in natural
    parameters: per term (sigma, omega0, Q) for SHO or (sigma, ell) for
    Matern-3/2, then the white-noise standard deviation ``s``.
    ``theta_per_series`` True means n_sets == n_series (set i for series i);
    False means every set is applied to every series.
    """

    name: str
    terms: list
    layout: int
    offsets: np.ndarray
    t_start: np.ndarray
    t_end: np.ndarray
    y: np.ndarray
    yerr: np.ndarray
    instrument: np.ndarray | None
    theta: np.ndarray
    theta_per_series: bool

    @property
    def n_series(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_meas(self) -> int:
        return int(self.offsets[-1])

    @property
    def n_params(self) -> int:
        return self.theta.shape[1]

    def series(self, i: int):
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        inst = None if self.instrument is None else self.instrument[a:b]
        return self.t_start[a:b], self.t_end[a:b], self.y[a:b], self.yerr[a:b], inst

    def with_theta(self, theta) -> "Workload":
        """The same series with other parameter sets (shared-set mode kept)."""
        return dataclasses.replace(self, theta=np.array(theta, dtype=np.float64, copy=True))

    def subset(self, idx) -> "Workload":
        """Workload restricted to the given series indices (theta follows)."""
        idx = np.asarray(idx, dtype=np.int64)
        parts = [np.arange(self.offsets[i], self.offsets[i + 1]) for i in idx]
        sel = np.concatenate(parts) if parts else np.zeros(0, np.int64)
        counts = np.array([self.offsets[i + 1] - self.offsets[i] for i in idx], np.int64)
        offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        th = self.theta[idx] if self.theta_per_series else self.theta
        return Workload(self.name, self.terms, self.layout, offs,
                        self.t_start[sel], self.t_end[sel], self.y[sel], self.yerr[sel],
                        None if self.instrument is None else self.instrument[sel],
                        th.copy(), self.theta_per_series)


def n_params_for(terms) -> int:
    return sum({SHO: 3, SHO_PRODUCT: 5}.get(k, 2) for k in terms) + 1


def _term_spectra(terms, theta_row):
    """(sigma, omega0, Q) of each term; Matern-3/2 is the Q = 1/2 oscillator;
    a product of two SHOs gives (sigma, omega_a, Q_a, omega_b, Q_b)."""
    out = []
    j = 0
    for k in terms:
        if k == SHO:
            out.append(tuple(theta_row[j:j + 3]))
            j += 3
        elif k == SHO_PRODUCT:
            out.append(tuple(theta_row[j:j + 5]))
            j += 5
        else:
            out.append((theta_row[j], math.sqrt(3.0) / theta_row[j + 1], 0.5))
            j += 2
    return out


def _rff(rng, t, sig, w0, q, n_feat):
    """Random-Fourier-feature draw with the oscillator's covariance at times t."""
    w = _sample_psd(rng, w0, q, n_feat)
    ph = rng.uniform(0, TWO_PI, n_feat)
    amp = sig * math.sqrt(2.0 / n_feat)
    out = np.zeros_like(t)
    for a in range(0, len(t), 16384):
        sl = slice(a, a + 16384)
        arg = np.mod(np.outer(t[sl], w) + ph, TWO_PI)
        out[sl] = amp * np.sum(np.cos(arg), axis=1)
    return out


def _sample_psd(rng, w0, q, n):
    """Angular frequencies drawn from the oscillator power spectrum
    S(w) ~ 1 / ((w^2 - w0^2)^2 + w0^2 w^2 / Q^2) (Eq. sho_psd), by inverse CDF
    on a log grid.  With random phases, sigma * sqrt(2/n) * sum cos(w t + p)
    then has covariance ~ k(t - t') (Bochner's theorem)."""
    w = w0 * np.logspace(-4, 4, 4001)
    dens = 1.0 / ((w * w - w0 * w0) ** 2 + (w0 * w / q) ** 2)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(w))])
    cdf /= cdf[-1]
    return np.interp(rng.uniform(0, 1, n), cdf, w)


def exposure_average_signal(rng, t_start, t_end, terms, theta_row, n_feat=16):
    """Exposure averages of a random-Fourier-feature draw of the kernel.

    Each term contributes ``n_feat`` cosines with random phases and angular
    frequencies drawn from that term's power spectrum, scaled to variance
    sigma^2.  The average of cos(w t + p) over [a, b] is
    cos(w (a+b)/2 + p) * sinc(w (b-a)/2), evaluated in that form so that
    short exposures do not cancel.
    """
    tm = 0.5 * (t_start + t_end)
    half = 0.5 * (t_end - t_start)
    f = np.zeros_like(tm)
    for par in _term_spectra(terms, theta_row):
        if len(par) == 5:
            # product of two independent draws: covariance sigma^2 k_a k_b
            # (instantaneous measurements only)
            if np.any(half != 0):
                raise NotImplementedError("product terms: instantaneous measurements only")
            sig, wa, qa, wb, qb = par
            f += _rff(rng, tm, 1.0, wa, qa, n_feat) * _rff(rng, tm, sig, wb, qb, n_feat)
            continue
        sig, w0, q = par
        w = _sample_psd(rng, w0, q, n_feat)
        ph = rng.uniform(0, TWO_PI, n_feat)
        amp = sig * math.sqrt(2.0 / n_feat)
        w32 = w.astype(np.float32)
        for a in range(0, len(tm), 16384):
            sl = slice(a, a + 16384)
            # phases reduced in FP64 before the FP32 cosine so long times keep their accuracy
            arg = np.mod(np.outer(tm[sl], w) + ph, TWO_PI).astype(np.float32)
            sinc = np.sinc(np.outer(half[sl].astype(np.float32), w32) / np.float32(math.pi))
            f[sl] += amp * np.sum(np.cos(arg) * sinc, axis=1, dtype=np.float64)
    return f


def single_instrument_exposures(rng, n, gap_mean, dmin, dmax, t0=0.0):
    """Start gaps ~ Exp(gap_mean); lengths ~ U[dmin, dmax] clipped to the gap."""
    gaps = rng.exponential(gap_mean, n)
    t_s = t0 + np.cumsum(gaps)
    dur = rng.uniform(dmin, dmax, n)
    nxt = np.empty(n)
    nxt[:-1] = t_s[1:] - t_s[:-1]
    nxt[-1] = np.inf
    dur = np.minimum(dur, nxt)
    t_e = t_s + dur
    # an exposure that ends exactly at the next start is allowed (no dead time)
    t_e[:-1] = np.minimum(t_e[:-1], t_s[1:])
    return t_s, t_e


def capped_overlap_exposures(rng, n, gap_mean, dmin, dmax, cap=3):
    """Exposures with at most ``cap`` open at once; returns (t_s, t_e, slot).

    Proposed starts follow cumulative Exp(gap_mean) gaps.  If ``cap``
    exposures are still open at a proposed start, the start is moved to the
    earliest open end and the new exposure takes that exposure's slot.
    """
    gaps = rng.exponential(gap_mean, n)
    dur = rng.uniform(dmin, dmax, n)
    t_s = np.empty(n)
    t_e = np.empty(n)
    slot = np.empty(n, np.int32)
    open_heap = []  # (end, slot)
    free = list(range(cap))
    t = 0.0
    for i in range(n):
        t += gaps[i]
        while open_heap and open_heap[0][0] <= t:
            _, s = heapq.heappop(open_heap)
            free.append(s)
        if not free:
            end, s = heapq.heappop(open_heap)
            t = max(t, end)
            free.append(s)
        free.sort()
        s = free.pop(0)
        t_s[i] = t
        t_e[i] = t + dur[i]
        slot[i] = s
        heapq.heappush(open_heap, (t_e[i], s))
    return t_s, t_e, slot


def _loguniform(rng, centre, factor, size=None):
    return centre * np.exp(rng.uniform(-0.5, 0.5, size) * math.log(factor))


def _finish(name, terms, layout, series, theta, theta_per_series, rng, s_white=0.1,
            with_instrument=False):
    """Concatenate per-series (t_s, t_e[, inst]) and draw y."""
    offs = [0]
    ts_all, te_all, y_all, inst_all = [], [], [], []
    for i, ser in enumerate(series):
        ts, te = ser[0], ser[1]
        row = theta[i] if theta_per_series else theta[0]
        f = exposure_average_signal(rng, ts, te, terms, row)
        y = f + s_white * rng.standard_normal(len(ts))
        ts_all.append(ts)
        te_all.append(te)
        y_all.append(y)
        if with_instrument:
            inst_all.append(ser[2].astype(np.int32))
        offs.append(offs[-1] + len(ts))
    t_s = np.concatenate(ts_all)
    t_e = np.concatenate(te_all)
    y = np.concatenate(y_all).astype(np.float32)
    yerr = np.zeros_like(y)
    inst = np.concatenate(inst_all) if with_instrument else None
    return Workload(name, list(terms), layout, np.asarray(offs, np.int64), t_s, t_e, y, yerr,
                    inst, np.asarray(theta, np.float64), theta_per_series)


def c1(seed=1001, n=1000):
    """One SHO series (omega0 = 2 pi/10, Q = 3, sigma = 1), s = 0.1."""
    rng = np.random.default_rng(seed)
    ts, te = single_instrument_exposures(rng, n, 1.0, 0.05, 0.5)
    theta = np.array([[1.0, TWO_PI / 10, 3.0, 0.1]])
    return _finish("c1", [SHO], 0, [(ts, te)], theta, True, rng)


def c2(seed=1002, n_series=4096, scale=1.0, nmin=500, nmax=20000):
    """Batched SHO + Matern-3/2 series with per-series parameters."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), n_series)) * scale)
    ns = np.maximum(ns, 2).astype(np.int64)
    theta = np.empty((n_series, 6))
    theta[:, 0] = _loguniform(rng, 1.0, 10, n_series)
    theta[:, 1] = _loguniform(rng, TWO_PI / 10, 10, n_series)
    theta[:, 2] = _loguniform(rng, 3.0, 10, n_series)
    theta[:, 3] = _loguniform(rng, 0.5, 10, n_series)
    theta[:, 4] = _loguniform(rng, 5.0, 10, n_series)
    theta[:, 5] = 0.1
    series = [single_instrument_exposures(rng, int(n), 1.0, 0.05, 0.5) for n in ns]
    return _finish("c2", [SHO, MATERN32], 0, series, theta, True, rng)


def c2i(seed=1006, n_series=4096, scale=1.0, nmin=500, nmax=20000, gap_mean=1.0):
    """The c2 recipe (SHO + Matern-3/2, per-series parameters log-uniform over
    a factor 10) on instantaneous measurements: times with Exponential(gap_mean)
    gaps, t_start == t_end, observing the latent itself (Section 2)."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), n_series)) * scale)
    ns = np.maximum(ns, 2).astype(np.int64)
    theta = np.empty((n_series, 6))
    theta[:, 0] = _loguniform(rng, 1.0, 10, n_series)
    theta[:, 1] = _loguniform(rng, TWO_PI / 10, 10, n_series)
    theta[:, 2] = _loguniform(rng, 3.0, 10, n_series)
    theta[:, 3] = _loguniform(rng, 0.5, 10, n_series)
    theta[:, 4] = _loguniform(rng, 5.0, 10, n_series)
    theta[:, 5] = 0.1
    series = []
    for n in ns:
        t = np.cumsum(rng.exponential(gap_mean, int(n)))
        series.append((t, t.copy()))
    return _finish("c2i", [SHO, MATERN32], 0, series, theta, True, rng)


def c2p(seed=1007, n_series=4096, scale=1.0, nmin=500, nmax=20000, gap_mean=1.0):
    """Quasi-periodic batch on instantaneous measurements: a product of two SHO
    terms (a slow envelope omega_a = 2 pi / 50, Q_a = 1 times a resonance
    omega_b = 2 pi / 5, Q_b = 10, Appendix C.2) plus a Matern-3/2 term, each
    parameter log-uniform over a factor 10 per series (Q_a truncated >= 0.55);
    times with Exponential(gap_mean) gaps."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), n_series)) * scale)
    ns = np.maximum(ns, 2).astype(np.int64)
    theta = np.empty((n_series, 8))
    theta[:, 0] = _loguniform(rng, 1.0, 10, n_series)
    theta[:, 1] = _loguniform(rng, TWO_PI / 50, 10, n_series)
    theta[:, 2] = np.maximum(_loguniform(rng, 1.0, 10, n_series), 0.55)
    theta[:, 3] = _loguniform(rng, TWO_PI / 5, 10, n_series)
    theta[:, 4] = _loguniform(rng, 10.0, 10, n_series)
    theta[:, 5] = _loguniform(rng, 0.5, 10, n_series)
    theta[:, 6] = _loguniform(rng, 5.0, 10, n_series)
    theta[:, 7] = 0.1
    series = []
    for n in ns:
        t = np.cumsum(rng.exponential(gap_mean, int(n)))
        series.append((t, t.copy()))
    return _finish("c2p", [SHO_PRODUCT, MATERN32], 0, series, theta, True, rng)


def c3(seed=1003, n=1 << 22):
    """One long series with up to 3 concurrently open exposures."""
    rng = np.random.default_rng(seed)
    ts, te, slot = capped_overlap_exposures(rng, n, 0.5, 0.5, 3.0, cap=3)
    theta = np.array([[1.0, TWO_PI / 10, 3.0, 0.1]])
    return _finish("c3", [SHO], 0, [(ts, te, slot)], theta, True, rng, with_instrument=True)


def c4(seed=1004, n_series=1024, scale=1.0, nmin=2000, nmax=20000):
    """Batched sum of two SHO terms; one integral state per term (layout 1)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, n_series)
    ns = np.maximum(np.rint(ns * scale), 2).astype(np.int64)
    theta = np.empty((n_series, 7))
    theta[:, 0] = _loguniform(rng, 1.0, 10, n_series)
    theta[:, 1] = _loguniform(rng, TWO_PI / 10, 10, n_series)
    theta[:, 2] = np.maximum(_loguniform(rng, 3.0, 10, n_series), 0.55)
    theta[:, 3] = _loguniform(rng, 0.5, 10, n_series)
    theta[:, 4] = _loguniform(rng, TWO_PI / 2, 10, n_series)
    theta[:, 5] = np.maximum(_loguniform(rng, 1.0, 10, n_series), 0.55)
    theta[:, 6] = 0.1
    series = [single_instrument_exposures(rng, int(n), 1.0, 0.05, 0.5) for n in ns]
    return _finish("c4", [SHO, SHO], 1, series, theta, True, rng)


def c5(seed=1005, n=1_000_000, n_sets=256):
    """One 3-instrument series shared by ``n_sets`` hyperparameter vectors."""
    rng = np.random.default_rng(seed)
    deltas = np.array([0.1, 1.0, 5.0])
    weights = 1.0 / deltas
    counts = np.floor(n * weights / weights.sum()).astype(np.int64)
    counts[0] += n - counts.sum()
    ts_l, te_l, in_l = [], [], []
    for i, (d, c) in enumerate(zip(deltas, counts)):
        gaps = d + rng.exponential(d, int(c))
        t_s = np.cumsum(gaps) - gaps[0]
        ts_l.append(t_s)
        te_l.append(t_s + d)
        in_l.append(np.full(int(c), i, np.int32))
    # interleave by start time, keeping each instrument's own order
    t_s = np.concatenate(ts_l)
    t_e = np.concatenate(te_l)
    inst = np.concatenate(in_l)
    order = np.argsort(t_s, kind="stable")
    t_s, t_e, inst = t_s[order], t_e[order], inst[order]
    centre = np.array([1.0, TWO_PI / 10, 3.0, 0.5, 5.0])
    th = np.exp(np.log(centre)[None, :] + 0.5 * rng.standard_normal((n_sets, 5)))
    th[:, 2] = np.maximum(th[:, 2], 0.55)
    theta = np.concatenate([th, np.full((n_sets, 1), 0.1)], axis=1)
    return _finish("c5", [SHO, MATERN32], 0, [(t_s, t_e, inst)], theta, False, rng,
                   with_instrument=True)


def mixed(seed, n_series, n, terms, theta_row, layout=0, frac_instant=0.5):
    """Series mixing exposure averages with instantaneous measurements (t_end
    == t_start): ``n`` exposures of the c1 recipe per series and about
    ``frac_instant * n`` instants drawn uniformly over the series' span, three
    of them placed on an exposure's start or end (simultaneous events)."""
    rng = np.random.default_rng(seed)
    series = []
    for _ in range(n_series):
        ts, te = single_instrument_exposures(rng, n, 1.0, 0.05, 0.5)
        ti = np.sort(rng.uniform(ts[0] - 1.0, te[-1] + 1.0, max(3, int(frac_instant * n))))
        ti[:3] = [ts[min(5, n - 1)], te[min(7, n - 1)], ts[min(9, n - 1)]]
        a = np.concatenate([ts, ti])
        b = np.concatenate([te, ti])
        series.append((a, b))
    theta = np.array([theta_row] * n_series, dtype=np.float64)
    return _finish("mixed", list(terms), layout, series, theta, True, rng)


def small_single(seed, n, terms, theta_row, gap_mean=1.0, dmin=0.05, dmax=0.5, s_white=0.1):
    """A one-series workload of the c1 exposure recipe with a given kernel."""
    rng = np.random.default_rng(seed)
    ts, te = single_instrument_exposures(rng, n, gap_mean, dmin, dmax)
    return _finish("single", list(terms), 0, [(ts, te)], np.asarray([theta_row], float), True,
                   rng, s_white=s_white)


def two_instrument_overlap(seed, n1, n2, d1=55.0, d2_mean=180.0, d2_sd=30.0, gap2=60.0,
                           sigma=1.0, timescale=300.0, q=3.0, s_white=0.3):
    """Two instruments in the shape of the paper's multi-instrument test:
    constant 55 s exposures back to back and 180 +- 30 s exposures, which
    frequently overlap (Section 4, Fig. 3).  Kernel: SHO with a ~300 s period."""
    rng = np.random.default_rng(seed)
    t1s = np.arange(n1) * d1
    t1e = t1s + d1
    d2 = np.clip(rng.normal(d2_mean, d2_sd, n2), 30.0, None)
    g2 = rng.exponential(gap2, n2)
    t2s = np.empty(n2)
    t = 0.0
    for i in range(n2):
        t += g2[i]
        t2s[i] = t
        t += d2[i]
    t2e = t2s + d2
    t_s = np.concatenate([t1s, t2s])
    t_e = np.concatenate([t1e, t2e])
    inst = np.concatenate([np.zeros(n1, np.int32), np.ones(n2, np.int32)])
    order = np.argsort(t_s, kind="stable")
    theta = np.array([[sigma, TWO_PI / timescale, q, s_white]])
    return _finish("two_inst", [SHO], 0, [(t_s[order], t_e[order], inst[order])], theta, True,
                   rng, s_white=s_white, with_instrument=True)

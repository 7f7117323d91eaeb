"""GPU parity of the conditioned mean and variance of every measurement's
exposure average (gp_ss_condition) against the oracle's integrated RTS
smoother (Eqs. rts, integrated_rts), which is pinned to the dense GP
posterior.

Tolerances (FP32 arithmetic, FP64 oracle), per series:
  mean      |a - b| <= 1e-3 max|mean| (+ 1e-5 relative to itself)
  variance  |a - b| <= 2e-3 |b| + 2e-4 v0, v0 the latent's prior variance
The posterior variance is a difference of prior-sized terms, so FP32 loses
about log10(prior / posterior) digits of it (gpu_checks).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_checks import check_mean_var, prior_var

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHO, M32 = 1, 2


@pytest.fixture(scope="module")
def gp():
    from paper_2601_02527_gb300 import build as gbuild
    gbuild.build()
    import paper_2601_02527_gb300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return g


def _f32(wl):
    wl.theta = wl.theta.astype(np.float32).astype(np.float64)
    return wl


_check = check_mean_var


def _oracle_cond(wl, s, theta):
    # (mean, variance, the latent's prior variance)
    ts, te, y, ye, inst = wl.series(s)
    mu, va = oracle.condition(wl.terms, wl.layout, ts, te, y, ye, theta, instrument=inst)
    return mu, va, prior_var(wl.terms, wl.layout, theta)


@pytest.mark.parametrize("chunk,ck", [(48, 8), (64, 16), (0, 32), (0, 64)])
def test_two_sho_layout1(gp, chunk, ck):
    wl = _f32(synth.c4(n_series=4, scale=0.05))
    m = gp.Model.from_workload(wl, chunk_len=chunk, ckpt_interval=ck)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    ll, cond = m.condition(th)
    ll_ref = m.loglik(th).cpu().numpy()
    np.testing.assert_allclose(ll.cpu().numpy(), ll_ref, rtol=1e-12)
    cond = cond.cpu().numpy()[0]
    for s in range(wl.n_series):
        a, b = wl.offsets[s], wl.offsets[s + 1]
        _check(cond[a:b], *_oracle_cond(wl, s, wl.theta[s]))


def test_three_overlapping_slots(gp):
    rng = np.random.default_rng(41)
    ts, te, slot = synth.capped_overlap_exposures(rng, 900, 0.5, 0.5, 3.0, cap=3)
    wl = _f32(synth._finish("c3s", [SHO], 0, [(ts, te, slot)],
                            np.array([[1.0, 2 * math.pi / 10, 3.0, 0.1]]), True, rng,
                            with_instrument=True))
    m = gp.Model.from_workload(wl, chunk_len=16, ckpt_interval=8)
    _, cond = m.condition(torch.tensor(wl.theta, dtype=torch.float32, device="cuda"))
    _check(cond.cpu().numpy()[0], *_oracle_cond(wl, 0, wl.theta[0]))


def test_shared_series_theta_sets(gp):
    # the three instruments all start at t = 0: their integral states are
    # reset together and stay equal, which the RTS recursion cannot invert;
    # the reference is the dense posterior (the plain definition)
    from oracle import dense
    wl = _f32(synth.c5(n=900, n_sets=3))
    m = gp.Model.from_workload(wl, chunk_len=32)
    _, cond = m.condition(torch.tensor(wl.theta, dtype=torch.float32, device="cuda"),
                          per_series=False)
    cond = cond.cpu().numpy()
    assert cond.shape == (3, wl.n_meas, 2)
    ts, te, y, ye, _ = wl.series(0)
    for k in range(3):
        _check(cond[k], *dense.posterior(wl.terms, wl.theta[k], ts, te, y, ye),
               prior_var(wl.terms, wl.layout, wl.theta[k]))


def test_edge_cases(gp):
    rng = np.random.default_rng(42)
    series = [(np.array([3.0]), np.array([3.2]))]           # one measurement
    ts = np.arange(80) * 0.5
    series.append((ts, ts + 0.5))                          # no dead time (exact ties)
    ts = np.cumsum(rng.exponential(1.0, 60))
    ts[30:] += 400.0                                       # a long gap
    series.append((ts, ts + 1e-3))
    series.append(synth.single_instrument_exposures(rng, 333, 1.0, 0.05, 0.5))
    theta = np.array([[1.0, 2 * math.pi / 10, 3.0, 0.1]] * len(series))
    wl = _f32(synth._finish("edge", [SHO], 0, series, theta, True, rng))
    for chunk in (0, 6, 64):
        m = gp.Model.from_workload(wl, chunk_len=chunk)
        _, cond = m.condition(torch.tensor(wl.theta, dtype=torch.float32, device="cuda"))
        cond = cond.cpu().numpy()[0]
        for s in range(wl.n_series):
            a, b = wl.offsets[s], wl.offsets[s + 1]
            _check(cond[a:b], *_oracle_cond(wl, s, wl.theta[s]))

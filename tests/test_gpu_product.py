"""GPU parity for product kernels (Appendix C.2) on instantaneous measurements
against the FP64 oracle: the plain per-series filter in FP32 (FP64 sums;
|L_gpu - L_or| <= 1e-4 max(|L_or|, 0.1 N)) and in FP64 (1e-9 relative), and
the forward-mode hyperparameter gradient, chunked and per series (1e-3 |g| +
1e-4 max|g| per component).
Calls the product path does not provide report GP_SS_EUNSUPPORTED.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHO, M32, PROD = 1, 2, 3


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


def _dev(th):
    return torch.tensor(th, dtype=torch.float32, device="cuda")


def _check(ll, ref, counts, rel=None):
    for a, b, n in zip(ll, ref, counts):
        tol = rel * abs(b) if rel else 1e-4 * max(abs(b), 0.1 * n)
        assert abs(a - b) <= tol, (a, b, n)


def _series_wl(terms, theta, n=600, seed=111):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(0.8, n))
    return _f32(synth._finish("p", terms, 0, [(t, t.copy())], np.asarray([theta]), True, rng))


@pytest.mark.parametrize("precision,schedule,chunk", [(32, 0, 0), (32, 2, 16), (32, 3, 0),
                                                     (64, 0, 0)])
def test_batch_product_plus_matern(gp, precision, schedule, chunk):
    # FP32: the chunked parallel-in-time path (product elements, shared
    # combination) at two chunk lengths, and the plain per-series filter
    wl = _f32(synth.c2p(n_series=8, scale=0.05))
    m = gp.Model.from_workload(wl, precision=precision, schedule=schedule, chunk_len=chunk)
    ll = m.loglik(_dev(wl.theta)).cpu().numpy()
    ref = oracle.loglik_workload(wl, processes=4)
    _check(ll, ref, np.diff(wl.offsets), rel=1e-9 if precision == 64 else None)
    assert m.last_error() == (-1, 0)


@pytest.mark.parametrize("terms,theta", [
    ([PROD], [1.2, 0.2, 1.5, 2.0, 8.0, 0.1]),
    ([PROD, SHO], [1.0, 0.3, 0.8, 1.3, 4.0, 0.6, 3.0, 0.3, 0.1]),   # overdamped plain term
    ([PROD], [0.9, 0.5, 0.3, 1.1, 2.0, 0.05])])                     # overdamped factor
def test_single_series(gp, terms, theta):
    wl = _series_wl(terms, theta)
    for precision, schedule, chunk in ((32, 0, 0), (32, 2, 8), (32, 3, 0), (64, 0, 0)):
        m = gp.Model.from_workload(wl, precision=precision, schedule=schedule, chunk_len=chunk)
        ll = m.loglik(_dev(wl.theta)).cpu().numpy()
        _check(ll, oracle.loglik_workload(wl), [wl.n_meas], rel=1e-9 if precision == 64 else None)


def _check_grad(g, ref_g):
    for a, b in zip(np.asarray(g, float), ref_g):
        bad = np.abs(a - b) > 1e-3 * np.abs(b) + 1e-4 * np.abs(b).max()
        assert not bad.any(), (a, b)


# (schedule, chunk length): the chunked forward-mode gradient (one thread per
# chunk and parameter, boundary adjoints from the combination) at the default
# and at a short chunk length, and the plain one (per series and parameter)
_GRAD_SCHEDULES = [(0, 0), (2, 8), (3, 0)]


@pytest.mark.parametrize("terms,theta", [
    ([PROD], [1.2, 0.2, 1.5, 2.0, 8.0, 0.1]),
    ([PROD, SHO], [1.0, 0.3, 0.8, 1.3, 4.0, 0.6, 3.0, 0.3, 0.1]),
    ([PROD, M32], [0.9, 0.5, 0.3, 1.1, 2.0, 0.5, 3.0, 0.05])])
def test_gradient(gp, terms, theta):
    # forward-mode tangents against the oracle's complex-step gradient
    wl = _series_wl(terms, theta, n=500)
    ref_ll, ref_g = oracle.loglik_workload(wl, grad=True)
    for schedule, chunk in _GRAD_SCHEDULES:
        m = gp.Model.from_workload(wl, schedule=schedule, chunk_len=chunk)
        ll, g = m.loglik_grad(_dev(wl.theta))
        _check(ll.cpu().numpy(), ref_ll, [wl.n_meas])
        _check_grad(g.cpu().numpy(), ref_g)
        assert m.last_error() == (-1, 0)


def test_gradient_batch(gp):
    wl = _f32(synth.c2p(n_series=12, scale=0.03))
    ref_ll, ref_g = oracle.loglik_workload(wl, grad=True, processes=4)
    got = {}
    for schedule, chunk in _GRAD_SCHEDULES:
        m = gp.Model.from_workload(wl, schedule=schedule, chunk_len=chunk)
        ll, g = m.loglik_grad(_dev(wl.theta))
        _check(ll.cpu().numpy(), ref_ll, np.diff(wl.offsets))
        _check_grad(g.cpu().numpy(), ref_g)
        got[schedule] = g.cpu().numpy().astype(float)
    # the chunked and the per-series tangents agree to FP32 rounding
    np.testing.assert_allclose(got[0], got[3], rtol=2e-4, atol=2e-5 * np.abs(got[3]).max())


def test_shared_theta_sets(gp):
    wl = _series_wl([PROD, M32], [1.0, 0.3, 1.0, 1.3, 5.0, 0.5, 3.0, 0.1], n=400)
    th = np.array([wl.theta[0], wl.theta[0] * [1, 1.2, 1, 0.9, 1, 1, 1, 1]], np.float64)
    th = th.astype(np.float32).astype(np.float64)
    m = gp.Model.from_workload(wl)
    ll = m.loglik(_dev(th), per_series=False).cpu().numpy().ravel()
    ref = [oracle.loglik(wl.terms, 0, *wl.series(0)[:4], th[k]) for k in range(2)]
    _check(ll, ref, [wl.n_meas] * 2)


def test_unsupported_calls(gp):
    wl = _series_wl([PROD], [1.2, 0.2, 1.5, 2.0, 8.0, 0.1], n=100)
    m = gp.Model.from_workload(wl)
    th = _dev(wl.theta)
    with pytest.raises(Exception):
        m.condition(th)
    with pytest.raises(Exception):
        m.loglik_grad(th, exposure=True)
    t = wl.t_start
    with pytest.raises(Exception):  # exposure averages with a product kernel
        gp.Model(wl.terms, wl.offsets, t, t + 0.1, wl.y, wl.yerr, None, layout=0)


def test_edge_cases(gp):
    rng = np.random.default_rng(112)
    t = np.cumsum(rng.exponential(1.0, 80))
    t[5:9] = t[5]          # repeated times
    t[40:] += 300.0        # one very long gap
    series = [np.array([1.5]), np.sort(t)]
    theta = np.array([[1.2, 0.2, 1.5, 2.0, 8.0, 0.1]] * 2)
    wl = _f32(synth._finish("pedge", [PROD], 0, [(s, s.copy()) for s in series], theta, True, rng))
    ref = oracle.loglik_workload(wl)
    for precision in (32, 64):
        ll = gp.Model.from_workload(wl, precision=precision).loglik(_dev(wl.theta)).cpu().numpy()
        _check(ll, ref, np.diff(wl.offsets), rel=1e-9 if precision == 64 else None)


@pytest.mark.parametrize("schedule,chunk", _GRAD_SCHEDULES)
def test_gradient_shared_sets_and_host_buffer(gp, schedule, chunk):
    wl = _series_wl([PROD, M32], [1.0, 0.3, 1.0, 1.3, 5.0, 0.5, 3.0, 0.1], n=300)
    th = np.array([wl.theta[0], wl.theta[0] * [1, 1.2, 1, 0.9, 1, 1, 1, 1]], np.float64)
    th = th.astype(np.float32).astype(np.float64)
    m = gp.Model.from_workload(wl, schedule=schedule, chunk_len=chunk)
    ll, g = m.loglik_grad(_dev(th), per_series=False)
    ll, g = ll.cpu().numpy().ravel(), g.cpu().numpy().reshape(2, -1)
    for k in range(2):
        r_ll, r_g = oracle.loglik(wl.terms, 0, *wl.series(0)[:4], th[k], grad=True)
        _check([ll[k]], [r_ll], [wl.n_meas])
        assert np.all(np.abs(g[k] - r_g) <= 1e-3 * np.abs(r_g) + 1e-4 * np.abs(r_g).max())
    ll_h, g_h = m.loglik_grad_host(wl.theta, reupload_events=True)
    ll_d, g_d = m.loglik_grad(_dev(wl.theta))
    np.testing.assert_array_equal(ll_d.cpu().numpy(), ll_h)
    np.testing.assert_array_equal(g_d.cpu().numpy(), g_h)

"""GPU parity for series of instantaneous measurements (t_start == t_end: the
plain SSM of Section 2, no integral states) against the FP64 oracle.

Tolerances as in the other parity tests (FP32 arithmetic, FP64 oracle):
loglik 1e-4 max(|L|, 0.1 N); gradients per component 1e-3 |g| + 1e-4 max|g|;
conditioned values and predictions as in test_gpu_condition.py.  The FP64
plain filter must match to 1e-9.
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


def _wl(n_series=8, scale=0.05, overdamped=False, seed=1006):
    wl = synth.c2i(seed=seed, n_series=n_series, scale=scale)
    if overdamped:
        wl.theta[::2, 2] = 0.3
    wl.theta = wl.theta.astype(np.float32).astype(np.float64)
    return wl


def _dev(th):
    return torch.tensor(th, dtype=torch.float32, device="cuda")


def _check_ll(got, ref, counts):
    for a, b, n in zip(got, ref, counts):
        assert abs(a - b) <= 1e-4 * max(abs(b), 0.1 * n), (a, b, n)


def _check_rows(got, ref):
    for a, b in zip(np.asarray(got, float), np.asarray(ref, float)):
        bad = np.abs(a - b) > 1e-3 * np.abs(b) + 1e-4 * np.max(np.abs(b))
        assert not bad.any(), (a, b)


def test_model_shape(gp):
    wl = _wl(n_series=3)
    m = gp.Model.from_workload(wl)
    assert m.info["n_slots"] == 0 and m.info["state_dim"] == 4
    assert m.info["n_events"] == wl.n_meas


def test_fp64_plain(gp):
    wl = _wl(n_series=4)
    m = gp.Model.from_workload(wl, precision=64)
    ll = m.loglik(_dev(wl.theta)).cpu().numpy()
    ref = oracle.loglik_workload(wl, processes=4)
    for a, b in zip(ll, ref):
        assert abs(a - b) <= 1e-9 * abs(b), (a, b)


@pytest.mark.parametrize("schedule,chunk", [(1, 0), (2, 64), (0, 0), (3, 0)])
@pytest.mark.parametrize("overdamped", [False, True])
def test_fp32_loglik(gp, schedule, chunk, overdamped):
    wl = _wl(n_series=10, scale=0.08, overdamped=overdamped)
    m = gp.Model.from_workload(wl, schedule=schedule, chunk_len=chunk)
    ll = m.loglik(_dev(wl.theta)).cpu().numpy()
    _check_ll(ll, oracle.loglik_workload(wl, processes=4), np.diff(wl.offsets))
    assert m.last_error() == (-1, 0)


@pytest.mark.parametrize("chunk,ck", [(48, 8), (0, 32), (64, 64)])
def test_gradient(gp, chunk, ck):
    wl = _wl(n_series=6, scale=0.05, overdamped=(ck == 8))
    m = gp.Model.from_workload(wl, chunk_len=chunk, ckpt_interval=ck)
    ll, g = m.loglik_grad(_dev(wl.theta))
    ref_ll, ref_g = oracle.loglik_workload(wl, grad=True, processes=4)
    _check_ll(ll.cpu().numpy(), ref_ll, np.diff(wl.offsets))
    _check_rows(g.cpu().numpy(), ref_g)


def test_time_gradient(gp):
    wl = _wl(n_series=3, scale=0.012)
    m = gp.Model.from_workload(wl, chunk_len=32, ckpt_interval=8)
    _, _, dexp = m.loglik_grad(_dev(wl.theta), exposure=True)
    dexp = dexp.cpu().numpy()[0]
    for s in range(wl.n_series):
        ts, te, y, ye, inst = wl.series(s)
        r_ts, r_te = oracle.exposure_grad(wl.terms, wl.layout, ts, te, y, ye, wl.theta[s])
        ref = np.stack([r_ts, r_te], axis=1)
        got = dexp[wl.offsets[s]:wl.offsets[s + 1]]
        bad = np.abs(got - ref) > 1e-3 * np.abs(ref) + 1e-4 * np.abs(ref).max()
        assert not bad.any(), (s, got[bad][:5], ref[bad][:5])


def test_condition_and_predict(gp):
    wl = _wl(n_series=4, scale=0.04)
    m = gp.Model.from_workload(wl, chunk_len=48, ckpt_interval=16)
    th = _dev(wl.theta)
    _, cond = m.condition(th)
    cond = cond.cpu().numpy()[0]
    rng = np.random.default_rng(91)
    tq, offs = [], [0]
    for s in range(wl.n_series):
        ts = wl.series(s)[0]
        q = np.concatenate([[ts.min() - 1.5], ts[::5], np.sort(rng.uniform(ts.min(), ts.max(), 60)),
                            [ts.max() + 0.4]])
        tq.append(q)
        offs.append(offs[-1] + len(q))
    tq, offs = np.concatenate(tq), np.array(offs, np.int64)
    _, pred = m.predict(th, tq, offs)
    pred = pred.cpu().numpy()[0]
    for s in range(wl.n_series):
        ts, te, y, ye, _ = wl.series(s)
        v0 = prior_var(wl.terms, wl.layout, wl.theta[s])
        for got, (mu, va) in (
                (cond[wl.offsets[s]:wl.offsets[s + 1]],
                 oracle.condition(wl.terms, wl.layout, ts, te, y, ye, wl.theta[s])),
                (pred[offs[s]:offs[s + 1]],
                 oracle.predict(wl.terms, wl.layout, ts, te, y, ye, wl.theta[s],
                                tq[offs[s]:offs[s + 1]]))):
            check_mean_var(got, mu, va, v0)


def test_single_term(gp):
    rng = np.random.default_rng(92)
    t = np.cumsum(rng.exponential(0.5, 700))
    th = np.array([[1.0, 2 * math.pi / 10, 3.0, 0.1]])
    wl = synth._finish("i1", [SHO], 0, [(t, t.copy())], th, True, rng)
    wl.theta = wl.theta.astype(np.float32).astype(np.float64)
    m = gp.Model.from_workload(wl, chunk_len=64)
    ll, g = m.loglik_grad(_dev(wl.theta))
    ref_ll, ref_g = oracle.loglik_workload(wl, grad=True)
    _check_ll(ll.cpu().numpy(), ref_ll, [len(t)])
    _check_rows(g.cpu().numpy(), ref_g)


def test_edge_cases(gp):
    rng = np.random.default_rng(93)
    series = []
    series.append(np.array([3.0]))                                   # single measurement
    t = np.cumsum(rng.exponential(1.0, 50))
    t[10:14] = t[10]                                                 # repeated times
    t[30:] += 500.0                                                  # one very long gap
    series.append(np.sort(t))
    series.append(np.zeros(0))                                       # empty series
    series.append(np.cumsum(rng.exponential(0.3, 333)))              # ragged length
    theta = np.array([[1.0, 2 * math.pi / 10, 3.0, 0.1]] * len(series))
    wl = synth._finish("iedge", [SHO], 0, [(s, s.copy()) for s in series], theta, True, rng)
    wl.theta = wl.theta.astype(np.float32).astype(np.float64)
    keep = [0, 1, 3]
    ref_ll, ref_g = oracle.loglik_workload(wl.subset(keep), grad=True)
    for chunk in (0, 7, 64):
        m = gp.Model.from_workload(wl, chunk_len=chunk)
        assert m.info["n_slots"] == 0  # the empty series asks for no integral state
        ll, g = m.loglik_grad(_dev(wl.theta))
        ll, g = ll.cpu().numpy(), g.cpu().numpy()
        assert ll[2] == 0.0 and np.all(g[2] == 0)
        _check_ll(ll[keep], ref_ll, np.diff(wl.offsets)[keep])
        _check_rows(g[keep], ref_g)


def test_host_buffer_and_shared_sets(gp):
    # the host-buffer call (grouped re-upload of the event stream) gives the
    # device call's bits; shared parameter sets against the oracle
    wl = _wl(n_series=6, scale=0.05)
    m = gp.Model.from_workload(wl, chunk_len=32)
    th = _dev(wl.theta)
    ll, g = m.loglik_grad(th)
    ll_h, g_h = m.loglik_grad_host(wl.theta, reupload_events=True)
    np.testing.assert_array_equal(ll.cpu().numpy(), ll_h)
    np.testing.assert_array_equal(g.cpu().numpy(), g_h)
    ll_s, g_s = m.loglik_grad(th[:2], per_series=False)
    ll_s = ll_s.cpu().numpy().reshape(2, wl.n_series)
    for k in range(2):
        ref_ll = [oracle.loglik(wl.terms, 0, *wl.series(i)[:4], wl.theta[k])
                  for i in range(wl.n_series)]
        _check_ll(ll_s[k], ref_ll, np.diff(wl.offsets))

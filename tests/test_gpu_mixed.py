"""GPU parity for models that mix exposure averages with instantaneous
measurements (t_end == t_start) in one series: the exposures keep their
integral states, the instants observe the latent (Section 2), and at equal
times the events go exposure ends, instants, starts.  Against the FP64
oracle, which handles mixed series (itself pinned to the dense GP in
test_oracle_instantaneous.py).

Tolerances as in test_gpu_parity.py: FP64 plain filter 1e-9; FP32
log-likelihood 1e-4 max(|L|, 0.1 N); gradients per component 1e-3 |g| +
1e-4 max|g|; conditioned values and predictions as in test_gpu_condition.py.
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
CASES = [([SHO], 0, [1.0, 0.7, 3.0, 0.1]),
         ([SHO, M32], 0, [1.0, 1.1, 2.0, 0.5, 3.0, 0.1]),
         ([SHO, SHO], 1, [1.0, 0.7, 3.0, 0.5, 2.0, 0.3, 0.1])]


@pytest.fixture(scope="module")
def gp():
    from paper_2601_02527_gb300 import build as gbuild
    gbuild.build()
    import paper_2601_02527_gb300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return g


def _wl(terms, layout, theta, n_series=3, n=150, seed=88):
    wl = synth.mixed(seed, n_series, n, terms, theta, layout=layout)
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


@pytest.mark.parametrize("terms,layout,theta", CASES)
def test_mixed_loglik_and_gradient(gp, terms, layout, theta):
    wl = _wl(terms, layout, theta)
    n_inst = int(np.sum(wl.t_end == wl.t_start))
    assert 0 < n_inst < wl.n_meas
    ref_ll, ref_g = oracle.loglik_workload(wl, grad=True)
    counts = np.diff(wl.offsets)
    m64 = gp.Model.from_workload(wl, precision=64)
    assert m64.info["n_events"] == 2 * wl.n_meas - n_inst and m64.info["n_slots"] >= 1
    l64 = m64.loglik(_dev(wl.theta)).cpu().numpy()
    assert np.all(np.abs(l64 - ref_ll) <= 1e-9 * np.abs(ref_ll)), (l64, ref_ll)
    for chunk, schedule in ((0, 0), (16, 2), (7, 2), (0, 3)):
        m = gp.Model.from_workload(wl, chunk_len=chunk, schedule=schedule)
        _check_ll(m.loglik(_dev(wl.theta)).cpu().numpy(), ref_ll, counts)
        if schedule != 3:
            ll, g = m.loglik_grad(_dev(wl.theta))
            _check_ll(ll.cpu().numpy(), ref_ll, counts)
            _check_rows(g.cpu().numpy(), ref_g)
            assert m.last_error() == (-1, 0)


def test_mixed_condition_predict_exposure(gp):
    terms, layout, theta = CASES[1]
    wl = _wl(terms, layout, theta, n_series=2, n=120, seed=89)
    m = gp.Model.from_workload(wl, chunk_len=24, ckpt_interval=16)
    th = _dev(wl.theta)
    _, cond = m.condition(th)
    cond = cond.cpu().numpy()[0].astype(np.float64)
    _, _, dexp = m.loglik_grad(th, exposure=True)
    dexp = dexp.cpu().numpy()[0].astype(np.float64)
    rng = np.random.default_rng(7)
    tq, offs = [], [0]
    for s in range(wl.n_series):
        ts = wl.series(s)[0]
        q = np.concatenate([[ts.min() - 1.0], np.sort(rng.uniform(ts.min(), ts.max(), 40)),
                            [ts.max() + 0.5]])
        tq.append(q)
        offs.append(offs[-1] + len(q))
    tq, offs = np.concatenate(tq), np.array(offs, np.int64)
    _, pred = m.predict(th, tq, offs)
    pred = pred.cpu().numpy()[0].astype(np.float64)
    for s in range(wl.n_series):
        a, b = wl.offsets[s], wl.offsets[s + 1]
        ts, te, y, ye, _ = wl.series(s)
        v0 = prior_var(wl.terms, wl.layout, wl.theta[s])
        check_mean_var(cond[a:b], *oracle.condition(wl.terms, wl.layout, ts, te, y, ye, wl.theta[s]),
                       v0)
        check_mean_var(pred[offs[s]:offs[s + 1]],
                       *oracle.predict(wl.terms, wl.layout, ts, te, y, ye, wl.theta[s],
                                       tq[offs[s]:offs[s + 1]]), v0)
        r_ts, r_te = oracle.exposure_grad(wl.terms, wl.layout, ts, te, y, ye, wl.theta[s])
        ref = np.stack([r_ts, r_te], axis=1)
        bad = np.abs(dexp[a:b] - ref) > 1e-3 * np.abs(ref) + 1e-4 * np.abs(ref).max()
        assert not bad.any(), (s, dexp[a:b][bad][:5], ref[bad][:5])


def test_mixed_host_buffer_and_noalloc(gp):
    terms, layout, theta = CASES[0]
    wl = _wl(terms, layout, theta, n_series=4, n=90, seed=90)
    m = gp.Model.from_workload(wl, chunk_len=16)
    th = _dev(wl.theta)
    ll, g = m.loglik_grad(th)
    ll_h, g_h = m.loglik_grad_host(wl.theta, reupload_events=True)
    np.testing.assert_array_equal(ll.cpu().numpy(), ll_h)
    np.testing.assert_array_equal(g.cpu().numpy(), g_h)
    lln = m.loglik_noalloc(th).cpu().numpy()
    _check_ll(lln, oracle.loglik_workload(wl), np.diff(wl.offsets))

"""GPU parity of the prediction at arbitrary times (gp_ss_predict) against the
oracle's Algorithm 1 (pinned to the dense GP prediction).

Test times: before the data, at the first event, every event time, inside
exposures and gaps, after the data.  Tolerances (FP32 arithmetic, FP64
oracle), per series: mean |a - b| <= 1e-3 max|mean| + 1e-5 |b|; variance
|a - b| <= 2e-3 |b| + 2e-4 v0, v0 the latent's prior variance (gpu_checks).
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


def _times(wl, rng):
    out, offs = [], [0]
    for s in range(wl.n_series):
        ts, te, _, _, _ = wl.series(s)
        inside = ts + rng.uniform(0, 1, len(ts)) * (te - ts)
        q = np.concatenate([[ts.min() - 2.0, ts.min()], ts, te, inside,
                            np.linspace(ts.min(), te.max(), 31), [te.max() + 0.7]])
        rng.shuffle(q)
        out.append(q)
        offs.append(offs[-1] + len(q))
    return np.concatenate(out), np.array(offs, np.int64)


_check = check_mean_var


@pytest.mark.parametrize("chunk,ck", [(32, 8), (0, 32), (64, 64)])
def test_two_sho_layout1(gp, chunk, ck):
    wl = _f32(synth.c4(n_series=3, scale=0.03))
    rng = np.random.default_rng(51)
    tq, offs = _times(wl, rng)
    m = gp.Model.from_workload(wl, chunk_len=chunk, ckpt_interval=ck)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    ll, pred = m.predict(th, tq, offs)
    np.testing.assert_allclose(ll.cpu().numpy(), m.loglik(th).cpu().numpy(), rtol=1e-12)
    pred = pred.cpu().numpy()[0]
    for s in range(wl.n_series):
        ts, te, y, ye, inst = wl.series(s)
        q = tq[offs[s]:offs[s + 1]]
        mu, va = oracle.predict(wl.terms, wl.layout, ts, te, y, ye, wl.theta[s], q)
        _check(pred[offs[s]:offs[s + 1]], mu, va,
               prior_var(wl.terms, wl.layout, wl.theta[s]))


def test_sho_plus_matern_overlap(gp):
    rng = np.random.default_rng(52)
    a = np.sort(rng.uniform(0, 60, 50))
    b = np.sort(rng.uniform(0.05, 60, 30))
    ts = np.concatenate([a, b])
    te = np.concatenate([np.minimum(a + rng.uniform(0.2, 1.5, 50), np.append(a[1:] - 1e-3, 99)),
                         np.minimum(b + rng.uniform(0.5, 2.5, 30), np.append(b[1:] - 1e-3, 99))])
    inst = np.concatenate([np.zeros(50, np.int32), np.ones(30, np.int32)])
    th = np.array([[1.0, 1.3, 2.0, 0.6, 4.0, 0.1]])
    wl = _f32(synth._finish("ov", [SHO, M32], 0, [(ts, te, inst)], th, True, rng,
                            with_instrument=True))
    tq, offs = _times(wl, rng)
    m = gp.Model.from_workload(wl, chunk_len=8, ckpt_interval=8)
    _, pred = m.predict(torch.tensor(wl.theta, dtype=torch.float32, device="cuda"), tq, offs)
    t0, t1, y, ye, ins = wl.series(0)
    _check(pred.cpu().numpy()[0], *oracle.predict(wl.terms, wl.layout, t0, t1, y, ye,
                                                  wl.theta[0], tq, instrument=ins),
           prior_var(wl.terms, wl.layout, wl.theta[0]))


def test_shared_series_sets(gp):
    wl = _f32(synth.c5(n=400, n_sets=2))
    rng = np.random.default_rng(53)
    tq, offs = _times(wl, rng)
    m = gp.Model.from_workload(wl, chunk_len=16)
    _, pred = m.predict(torch.tensor(wl.theta, dtype=torch.float32, device="cuda"), tq, offs,
                        per_series=False)
    pred = pred.cpu().numpy()
    from oracle import dense
    t0, t1, y, ye, _ = wl.series(0)
    for k in range(2):
        # coincident resets at t = 0: the dense prediction is the reference
        _check(pred[k], *dense.predict(wl.terms, wl.theta[k], t0, t1, y, ye, tq),
               prior_var(wl.terms, wl.layout, wl.theta[k]))

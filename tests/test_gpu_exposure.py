"""GPU parity of the exposure-window gradient (d loglik / d t_start, d t_end
per measurement) against the oracle's complex-step derivative.

Tolerance as for the hyperparameter gradient (FP32 arithmetic, FP64 oracle):
per series, |g_gpu - g_or| <= 1e-3 |g_or| + 1e-4 max|g_or| elementwise.
Series are test-sized because the oracle needs one complex filter pass per
window edge.
"""
import math

import numpy as np
import pytest

import oracle
import synth

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


def _oracle_exp(wl, s, theta):
    ts, te, y, ye, inst = wl.series(s)
    return oracle.exposure_grad(wl.terms, wl.layout, ts, te, y, ye, theta, instrument=inst)


def _check(got, ref_ts, ref_te):
    ref = np.stack([ref_ts, ref_te], axis=1)
    scale = np.abs(ref).max()
    bad = np.abs(got - ref) > 1e-3 * np.abs(ref) + 1e-4 * scale
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], ref[bad][:5])


def _f32(wl):
    wl.theta = wl.theta.astype(np.float32).astype(np.float64)
    return wl


@pytest.mark.parametrize("chunk,ck,cache", [(48, 8, 0), (64, 16, 0), (0, 32, 0), (48, 16, 1)])
def test_two_sho_layout1(gp, chunk, ck, cache):
    wl = _f32(synth.c4(n_series=3, scale=0.012))
    m = gp.Model.from_workload(wl, chunk_len=chunk, ckpt_interval=ck, step_cache=cache)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    ll, g, dexp = m.loglik_grad(th, exposure=True)
    ll2, g2 = m.loglik_grad(th)
    # the call with exposure gradients runs a separately compiled kernel body:
    # the same arithmetic up to FP32 rounding order
    np.testing.assert_array_equal(ll.cpu().numpy(), ll2.cpu().numpy())
    np.testing.assert_allclose(g.cpu().numpy(), g2.cpu().numpy(), rtol=1e-5,
                               atol=1e-6 * np.abs(g2.cpu().numpy()).max())
    dexp = dexp.cpu().numpy()[0]
    for s in range(wl.n_series):
        a, b = wl.offsets[s], wl.offsets[s + 1]
        _check(dexp[a:b], *_oracle_exp(wl, s, wl.theta[s]))


def test_three_overlapping_slots(gp):
    rng = np.random.default_rng(31)
    ts, te, slot = synth.capped_overlap_exposures(rng, 120, 0.5, 0.5, 3.0, cap=3)
    wl = _f32(synth._finish("c3s", [SHO], 0, [(ts, te, slot)],
                            np.array([[1.0, 2 * math.pi / 10, 3.0, 0.1]]), True, rng,
                            with_instrument=True))
    m = gp.Model.from_workload(wl, chunk_len=8, ckpt_interval=8)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    _, _, dexp = m.loglik_grad(th, exposure=True)
    _check(dexp.cpu().numpy()[0], *_oracle_exp(wl, 0, wl.theta[0]))


def test_shared_series_theta_sets(gp):
    wl = _f32(synth.c5(n=150, n_sets=3))
    m = gp.Model.from_workload(wl, chunk_len=16, ckpt_interval=8)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    _, _, dexp = m.loglik_grad(th, per_series=False, exposure=True)
    dexp = dexp.cpu().numpy()
    assert dexp.shape == (3, wl.n_meas, 2)
    for k in range(3):
        _check(dexp[k], *_oracle_exp(wl, 0, wl.theta[k]))


def test_time_shift_invariance_on_gpu(gp):
    # a stationary kernel: moving every window together changes nothing
    wl = _f32(synth.c4(n_series=4, scale=0.05))
    m = gp.Model.from_workload(wl)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    _, _, dexp = m.loglik_grad(th, exposure=True)
    d = dexp.cpu().numpy()[0].astype(np.float64)
    for s in range(wl.n_series):
        a, b = wl.offsets[s], wl.offsets[s + 1]
        tot = d[a:b].sum()
        assert abs(tot) <= 1e-4 * np.abs(d[a:b]).sum(), (s, tot)


@pytest.mark.parametrize("per_series", [True, False])
def test_autograd_windows(gp, per_series):
    if per_series:
        wl = _f32(synth.c4(n_series=3, scale=0.02))
        th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    else:
        wl = _f32(synth.c5(n=300, n_sets=4))
        th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    m = gp.Model.from_workload(wl, chunk_len=32)
    win = torch.tensor(np.stack([wl.t_start, wl.t_end], axis=1), device="cuda",
                       dtype=torch.float64, requires_grad=True)
    thv = th.clone().requires_grad_(True)
    ll = gp.loglik(m, thv, per_series=per_series, windows=win)
    wts = torch.linspace(0.5, 1.5, ll.numel(), dtype=torch.float64, device="cuda")
    (ll * wts).sum().backward()
    _, g, dexp = m.loglik_grad(th, per_series=per_series, exposure=True)
    w32 = wts.float()
    if per_series:
        sidx = m.measurement_series("cuda")
        ref = w32[sidx][:, None] * dexp[0]
        gref = w32[:, None] * g
    else:
        sidx = m.measurement_series("cuda")
        coef = w32.view(th.shape[0], wl.n_series)[:, sidx]
        ref = (coef[:, :, None] * dexp).sum(0)
        gref = (w32[:, None] * g).view(th.shape[0], wl.n_series, -1).sum(1)
    np.testing.assert_allclose(win.grad.cpu().numpy(), ref.double().cpu().numpy(), rtol=1e-6)
    np.testing.assert_allclose(thv.grad.cpu().numpy(), gref.cpu().numpy(), rtol=1e-6)

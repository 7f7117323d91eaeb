"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (stated for FP32 arithmetic with FP64 log-likelihood sums):
  * FP64 plain filter: |L_gpu - L_or| <= 1e-9 |L_or|.
  * FP32 log-likelihood: |L_gpu - L_or| <= 1e-4 max(|L_or|, 0.1 N).
  * FP32 gradient, per component i of a series' gradient g:
        |g_gpu,i - g_or,i| <= 1e-3 |g_or,i| + 1e-4 ||g_or||_inf.
  * discretisation entries: |a - b| <= 2e-5 |b| + 2e-6 max|B|.
Sizes span several chunks and ragged tails; the full-size checks are in
test_gpu_fullsize.py.
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


def ll_tol(ll_or, n):
    return 1e-4 * max(abs(ll_or), 0.1 * n)


def check_ll(ll_gpu, ll_or, counts):
    for a, b, n in zip(ll_gpu, ll_or, counts):
        assert abs(a - b) <= ll_tol(b, n), (a, b, n)


def check_grad(g_gpu, g_or):
    g_gpu = np.asarray(g_gpu, float)
    g_or = np.asarray(g_or, float)
    for a, b in zip(g_gpu, g_or):
        scale = np.max(np.abs(b))
        bad = np.abs(a - b) > 1e-3 * np.abs(b) + 1e-4 * scale
        assert not bad.any(), (a, b)


def counts_of(wl):
    return np.diff(wl.offsets)


def oracle_ll(wl, grad=False):
    return oracle.loglik_workload(wl, grad=grad, processes=4)


def theta_dev(wl):
    return torch.tensor(wl.theta, dtype=torch.float32, device="cuda")


def f32_theta(wl):
    """The oracle sees exactly the FP32-rounded parameters the GPU gets."""
    wl.theta = wl.theta.astype(np.float32).astype(np.float64)
    return wl


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("terms,layout,n_slots,theta", [
    ([SHO], 0, 1, [1.0, 2 * math.pi / 10, 3.0, 0.1]),
    ([SHO], 0, 3, [0.7, 2.0, 0.8, 0.1]),
    ([M32], 0, 1, [0.5, 5.0, 0.1]),
    ([SHO, M32], 0, 2, [1.0, 0.9, 9.0, 0.5, 2.0, 0.1]),
    ([SHO, SHO], 1, 1, [1.0, 0.63, 3.0, 0.5, 3.1, 0.6, 0.1])])
def test_discretization_grid(gp, terms, layout, n_slots, theta):
    th32 = np.asarray(theta, np.float32)
    dts = np.concatenate([[0.0], np.logspace(-6, np.log10(60.0), 301)]).astype(np.float32)
    phi, q = gp.discretize(terms, layout, n_slots, torch.tensor(th32, device="cuda"),
                           torch.tensor(dts, device="cuda"))
    phi, q = phi.cpu().numpy(), q.cpu().numpy()
    for k, dt in enumerate(dts):
        P, Q, _ = oracle.discretize(terms, layout, n_slots, th32.astype(np.float64), float(dt))
        for got, ref in ((phi[k], P), (q[k], Q)):
            scale = np.max(np.abs(ref))
            ok = np.abs(got - ref) <= 2e-5 * np.abs(ref) + 2e-6 * scale
            assert ok.all(), (dt, got, ref)


def test_plain_fp64_matches_oracle_c1(gp):
    wl = f32_theta(synth.c1())
    m = gp.Model.from_workload(wl, precision=64)
    ll = m.loglik(theta_dev(wl)).cpu().numpy()
    ref = oracle_ll(wl)
    assert abs(ll[0] - ref[0]) <= 1e-9 * abs(ref[0]), (ll, ref)


@pytest.mark.parametrize("schedule,chunk", [(1, 0), (2, 64), (2, 200), (0, 0), (3, 0)])
def test_fp32_batch_loglik(gp, schedule, chunk):
    wl = f32_theta(synth.c2(n_series=12, scale=0.08))
    m = gp.Model.from_workload(wl, schedule=schedule, chunk_len=chunk)
    ll = m.loglik(theta_dev(wl)).cpu().numpy()
    check_ll(ll, oracle_ll(wl), counts_of(wl))
    assert m.last_error() == (-1, 0)


def test_fp32_plain_per_series_kernel_matches(gp):
    wl = f32_theta(synth.c2(n_series=6, scale=0.05))
    m64 = gp.Model.from_workload(wl, precision=64)
    m32 = gp.Model.from_workload(wl)
    a = m64.loglik(theta_dev(wl)).cpu().numpy()
    b = m32.loglik(theta_dev(wl)).cpu().numpy()
    ref = oracle_ll(wl)
    for x, y, n in zip(a, ref, counts_of(wl)):
        assert abs(x - y) <= 1e-9 * abs(y)
    check_ll(b, ref, counts_of(wl))


@pytest.mark.parametrize("chunk,combine", [(8, 2), (8, 1), (48, 0), (256, 0)])
def test_fp32_grad_layout1(gp, chunk, combine):
    wl = f32_theta(synth.c4(n_series=6, scale=0.05))
    m = gp.Model.from_workload(wl, chunk_len=chunk, combine=combine)
    ll, g = m.loglik_grad(theta_dev(wl))
    ref_ll, ref_g = oracle_ll(wl, grad=True)
    check_ll(ll.cpu().numpy(), ref_ll, counts_of(wl))
    check_grad(g.cpu().numpy(), ref_g)
    # the gradient path returns the same log-likelihood as the plain call
    ll2 = m.loglik(theta_dev(wl)).cpu().numpy()
    np.testing.assert_allclose(ll.cpu().numpy(), ll2, rtol=1e-12)


@pytest.mark.parametrize("ck", [8, 16, 32, 64])
def test_step_cache_off_matches(gp, ck):
    # the reverse sweep recomputing the step scalars gives the gradient of
    # the cached path (same FP32 arithmetic up to contraction) and the oracle's
    wl = f32_theta(synth.c4(n_series=6, scale=0.05))
    th = theta_dev(wl)
    on = gp.Model.from_workload(wl, chunk_len=48, ckpt_interval=ck)
    off = gp.Model.from_workload(wl, chunk_len=48, ckpt_interval=ck, step_cache=1)
    ll_a, g_a = on.loglik_grad(th)
    ll_b, g_b = off.loglik_grad(th)
    np.testing.assert_array_equal(ll_a.cpu().numpy(), ll_b.cpu().numpy())
    g_a, g_b = g_a.cpu().numpy(), g_b.cpu().numpy()
    assert np.all(np.abs(g_a - g_b) <= 1e-5 * np.abs(g_a) + 1e-6 * np.abs(g_a).max())
    _, ref_g = oracle_ll(wl, grad=True)
    check_grad(g_b, ref_g)


@pytest.mark.parametrize("chunk", [4, 8, 40, 300])
def test_overlapping_three_slots(gp, chunk):
    rng = np.random.default_rng(77)
    ts, te, slot = synth.capped_overlap_exposures(rng, 1500, 0.5, 0.5, 3.0, cap=3)
    wl = synth._finish("c3s", [SHO], 0, [(ts, te, slot)],
                       np.array([[1.0, 2 * math.pi / 10, 3.0, 0.1]]), True, rng,
                       with_instrument=True)
    wl = f32_theta(wl)
    m = gp.Model.from_workload(wl, chunk_len=chunk)
    assert m.info["n_slots"] == 3 and m.info["state_dim"] == 5
    ll, g = m.loglik_grad(theta_dev(wl))
    ref_ll, ref_g = oracle_ll(wl, grad=True)
    check_ll(ll.cpu().numpy(), ref_ll, counts_of(wl))
    check_grad(g.cpu().numpy(), ref_g)


@pytest.mark.parametrize("chunk", [4, 16, 128])
def test_theta_sets_shared_series(gp, chunk):
    wl = synth.c5(n=1200, n_sets=5)
    wl = f32_theta(wl)
    m = gp.Model.from_workload(wl, chunk_len=chunk)
    assert m.info["state_dim"] == 7
    th = theta_dev(wl)
    ll, g = m.loglik_grad(th, per_series=False)
    ref_ll, ref_g = oracle_ll(wl, grad=True)
    check_ll(ll.cpu().numpy(), ref_ll, [wl.n_meas] * len(ref_ll))
    check_grad(g.cpu().numpy(), ref_g)


def test_sho_plus_matern_grad(gp):
    wl = f32_theta(synth.c2(n_series=5, scale=0.05))
    m = gp.Model.from_workload(wl, chunk_len=100)
    ll, g = m.loglik_grad(theta_dev(wl))
    ref_ll, ref_g = oracle_ll(wl, grad=True)
    check_ll(ll.cpu().numpy(), ref_ll, counts_of(wl))
    check_grad(g.cpu().numpy(), ref_g)


def test_edge_cases(gp):
    rng = np.random.default_rng(5)
    series = []
    # single measurement
    series.append((np.array([3.0]), np.array([3.2])))
    # zero dead time
    ts = np.arange(60) * 0.4
    series.append((ts, ts + 0.4))
    # very short exposures and one very long gap
    ts = np.cumsum(rng.exponential(1.0, 50))
    ts[25:] += 400.0
    series.append((ts, ts + 1e-4))
    # one ordinary series with a ragged number of events
    series.append(synth.single_instrument_exposures(rng, 333, 1.0, 0.05, 0.5))
    theta = np.array([[1.0, 2 * math.pi / 10, 3.0, 0.1]] * len(series))
    wl = f32_theta(synth._finish("edge", [SHO], 0, series, theta, True, rng))
    for chunk in (0, 7, 64):
        m = gp.Model.from_workload(wl, chunk_len=chunk)
        ll, g = m.loglik_grad(theta_dev(wl))
        ref_ll, ref_g = oracle_ll(wl, grad=True)
        check_ll(ll.cpu().numpy(), ref_ll, counts_of(wl))
        check_grad(g.cpu().numpy(), ref_g)


def test_empty_series_in_batch(gp):
    rng = np.random.default_rng(9)
    a = synth.single_instrument_exposures(rng, 40, 1.0, 0.05, 0.5)
    b = (np.zeros(0), np.zeros(0))
    theta = np.array([[1.0, 0.7, 2.0, 0.1]] * 3)
    wl = f32_theta(synth._finish("empty", [SHO], 0, [a, b, a], theta, True, rng))
    m = gp.Model.from_workload(wl, chunk_len=16)
    ll, g = m.loglik_grad(theta_dev(wl))
    ll = ll.cpu().numpy()
    assert ll[1] == 0.0 and np.all(g.cpu().numpy()[1] == 0)
    ref = oracle.loglik_workload(wl.subset([0, 2]))
    check_ll(ll[[0, 2]], ref, [40, 40])


def test_graph_and_host_paths_agree(gp):
    wl = f32_theta(synth.c4(n_series=5, scale=0.03))
    m = gp.Model.from_workload(wl, chunk_len=96)
    th = theta_dev(wl)
    n0 = gp.launch_count()
    ll, g = m.loglik_grad(th)
    # tables, elements, combination (>= 3), finish, gradient, per-series sums
    assert gp.launch_count() - n0 >= 8
    for _ in range(2):
        ll_b, g_b = m.loglik_grad(th, batched=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ll.cpu().numpy(), ll_b.cpu().numpy())
        np.testing.assert_array_equal(g.cpu().numpy(), g_b.cpu().numpy())
    ll_l = m.loglik(th, batched=True)
    np.testing.assert_array_equal(ll.cpu().numpy(), ll_l.cpu().numpy())
    ll_h, g_h = m.loglik_grad_host(wl.theta, reupload_events=True)
    np.testing.assert_array_equal(ll.cpu().numpy(), ll_h)
    np.testing.assert_array_equal(g.cpu().numpy(), g_h)
    # shared parameter sets: the event stream re-sent in series groups whose
    # element passes start as each group arrives gives the same bits
    th2 = th[:3]
    ll_s, g_s = m.loglik_grad(th2, per_series=False)
    ll_hs, g_hs = m.loglik_grad_host(wl.theta[:3], per_series=False, reupload_events=True)
    np.testing.assert_array_equal(ll_s.cpu().numpy().ravel(), ll_hs.ravel())
    np.testing.assert_array_equal(g_s.cpu().numpy().reshape(g_hs.shape), g_hs)


def test_autograd_function(gp):
    wl = f32_theta(synth.c4(n_series=3, scale=0.03))
    m = gp.Model.from_workload(wl)
    th = theta_dev(wl).requires_grad_(True)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")
    (gp.loglik(m, th) * w).sum().backward()
    _, g = m.loglik_grad(th.detach())
    np.testing.assert_allclose(th.grad.cpu().numpy(),
                               (g * w.float()[:, None]).cpu().numpy(), rtol=1e-6)


def test_numeric_failure_is_reported(gp):
    wl = f32_theta(synth.c4(n_series=4, scale=0.02))
    m = gp.Model.from_workload(wl)
    th = theta_dev(wl)
    th[2, 2] = float("nan")  # a non-finite parameter -> non-finite innovation variances
    m.loglik(th)
    torch.cuda.synchronize()
    row, code = m.last_error()
    assert row == 2 and code == 7
    m.loglik(theta_dev(wl))
    torch.cuda.synchronize()
    assert m.last_error() == (-1, 0)


def test_autotune_gradient(gp):
    wl = f32_theta(synth.c4(n_series=6, scale=0.05))
    m = gp.Model.from_workload(wl)
    th = theta_dev(wl)
    best = m.autotune(th, grad=True, reps=1)
    assert best["schedule"] in (1, 2) and best["ckpt_interval"] in (16, 32, 64)
    assert best["n_tried"] >= 10 and best["ms"] > 0
    assert m.info["n_chunks"] >= 32 * wl.n_series
    ll, g = m.loglik_grad(th)
    ref_ll, ref_g = oracle_ll(wl, grad=True)
    check_ll(ll.cpu().numpy(), ref_ll, counts_of(wl))
    check_grad(g.cpu().numpy(), ref_g)


def test_autotune_loglik(gp):
    wl = f32_theta(synth.c2(n_series=12, scale=0.08))
    m = gp.Model.from_workload(wl)
    th = theta_dev(wl)
    best = m.autotune(th, grad=False, reps=1)
    assert best["schedule"] in (1, 2, 3)
    check_ll(m.loglik(th).cpu().numpy(), oracle_ll(wl), counts_of(wl))
    # a gradient call after a log-likelihood tuning still works
    _, g = m.loglik_grad(th)
    assert np.isfinite(g.cpu().numpy()).all()


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("combine,chunk", [(1, 24), (2, 24), (2, 8)])
def test_combination_precision(gp, prec, combine, chunk):
    # the cross-chunk combination in FP32 or FP64 (sequential fold or warp
    # scans + fold/scan of warp totals): log-likelihood and gradient against
    # the oracle, per-series and shared-set modes
    wl = f32_theta(synth.c4(n_series=5, scale=0.04))
    m = gp.Model.from_workload(wl, chunk_len=chunk, combine=combine, combine_precision=prec)
    ll, g = m.loglik_grad(theta_dev(wl))
    ref_ll, ref_g = oracle_ll(wl, grad=True)
    check_ll(ll.cpu().numpy(), ref_ll, counts_of(wl))
    check_grad(g.cpu().numpy(), ref_g)
    np.testing.assert_allclose(m.loglik(theta_dev(wl)).cpu().numpy(), ll.cpu().numpy(),
                               rtol=1e-12)
    ws = f32_theta(synth.c5(n=900, n_sets=3))
    ms = gp.Model.from_workload(ws, chunk_len=chunk, combine=combine, combine_precision=prec)
    lls, gs = ms.loglik_grad(theta_dev(ws), per_series=False)
    ref_ll, ref_g = oracle_ll(ws, grad=True)
    check_ll(lls.cpu().numpy(), ref_ll, [ws.n_meas] * len(ref_ll))
    check_grad(gs.cpu().numpy(), ref_g)
    # the no-allocation path follows the model's combination precision
    lln = ms.loglik_noalloc(theta_dev(ws), per_series=False).cpu().numpy()
    check_ll(lln, ref_ll, [ws.n_meas] * len(ref_ll))


def test_output_buffers_are_checked(gp):
    wl = f32_theta(synth.c4(n_series=3, scale=0.02))
    m = gp.Model.from_workload(wl)
    th = theta_dev(wl)
    with pytest.raises(ValueError):
        m.loglik(th, out=torch.empty(3, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        m.loglik(th, out=torch.empty(2, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        m.loglik_grad(th, grad=torch.empty(3, m.n_params, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        m.loglik(th, out=torch.empty(6, dtype=torch.float64, device="cuda")[::2])

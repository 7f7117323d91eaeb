"""A single series split in time across ranks, on one GPU: the ranks are
emulated by calling gp_ss_span_element for each rank's chunk range in turn
(no rank waits on another: the exchange is the host's stacking of the
elements, standing in for the all-gather), then gp_ss_span_loglik folds them.
The result must be the unsplit log-likelihood: against the model's own
gp_ss_loglik (FP32 tolerance), the FP64 plain filter and the oracle.
Tolerances as in test_gpu_parity.py: 1e-4 max(|L|, 0.1 N)."""
import numpy as np
import pytest

import oracle
import synth
from paper_2601_02527_gb300 import shard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    from paper_2601_02527_gb300 import build as gbuild
    gbuild.build()
    import paper_2601_02527_gb300 as g
    assert torch.cuda.is_available()
    oracle.build()
    return g


def _prefix(wl, n, sets=None):
    ts, te, y, ye, inst = wl.series(0)
    th = wl.theta if sets is None else wl.theta[sets]
    per = sets is None
    out = synth.Workload(wl.name + "p", wl.terms, wl.layout, np.array([0, n]), ts[:n], te[:n],
                         y[:n], ye[:n], inst[:n], th, per)
    out.theta = out.theta.astype(np.float32).astype(np.float64)
    return out


def _split(gp, m, th, world, per_series):
    ranges = shard.span_chunk_ranges(m.info["n_chunks"], world)
    elems = torch.stack([m.span_element(th, c0, c1, per_series=per_series) for c0, c1 in ranges])
    return m.span_loglik(elems).cpu().numpy()


@pytest.mark.parametrize("world", [1, 2, 3, 8])
@pytest.mark.parametrize("chunk", [16, 64])
def test_c3_prefix_split_in_time(gp, world, chunk):
    wl = _prefix(synth.c3(n=1 << 16), 1 << 16)
    m = gp.Model.from_workload(wl, chunk_len=chunk)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    got = _split(gp, m, th, world, True)
    ref = m.loglik(th).cpu().numpy()
    tol = 1e-4 * max(abs(ref[0]), 0.1 * wl.n_meas)
    assert abs(got[0] - ref[0]) <= tol, (got, ref)
    l64 = gp.Model.from_workload(wl, precision=64).loglik(th).cpu().numpy()
    assert abs(got[0] - l64[0]) <= tol, (got, l64)
    assert m.last_error() == (-1, 0)


def test_small_split_vs_oracle(gp):
    wl = _prefix(synth.c3(n=4000), 4000)
    m = gp.Model.from_workload(wl, chunk_len=8)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    ref = oracle.loglik_workload(wl)
    for world in (2, 5):
        got = _split(gp, m, th, world, True)
        assert abs(got[0] - ref[0]) <= 1e-4 * max(abs(ref[0]), 0.1 * wl.n_meas), (got, ref)


def test_shared_sets_split_in_time(gp):
    # the c5 recipe (three instruments, shared parameter sets): one row per set
    wl = _prefix(synth.c5(n=30000, n_sets=6), 30000, sets=np.arange(6))
    m = gp.Model.from_workload(wl, chunk_len=32)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    ref = m.loglik(th, per_series=False).cpu().numpy()
    for world in (2, 4):
        got = _split(gp, m, th, world, False)
        tol = 1e-4 * np.maximum(np.abs(ref), 0.1 * wl.n_meas)
        assert np.all(np.abs(got - ref) <= tol), (got, ref)


def test_span_arguments_checked(gp):
    wl = synth.c2(n_series=3, scale=0.02)
    m = gp.Model.from_workload(wl)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    with pytest.raises(gp.GPSSError) as e:
        m.span_element(th, 0, 32)
    assert e.value.code == 4  # more than one series
    w1 = _prefix(synth.c3(n=3000), 3000)
    m1 = gp.Model.from_workload(w1, chunk_len=16)
    t1 = torch.tensor(w1.theta, dtype=torch.float32, device="cuda")
    for c0, c1 in ((0, 0), (5, 3), (0, m1.info["n_chunks"] + 1), (-1, 4)):
        with pytest.raises(gp.GPSSError) as e:
            m1.span_element(t1, c0, c1)
        assert e.value.code == 1

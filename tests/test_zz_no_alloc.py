"""gp_ss_loglik_noalloc: the log-likelihood entry point that allocates no
device memory, for callers that cannot allocate at call time (their device
memory belongs to their own pool, or an allocation's latency or
synchronisation is not acceptable where they call).  Its scratch is one fixed
16 MiB array per GPU inside the library.

Checked through the C ABI: two calls in a row give the same values as
gp_ss_loglik within the FP32 log-likelihood tolerance of the parity tests
(|a - b| <= 1e-4 max(|b|, 0.1 N)), and a problem larger than the fixed array
is refused with GP_SS_ETOOBIG.  This file is collected last on purpose."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    from paper_2601_02527_gb300 import build as gbuild
    gbuild.build()
    import paper_2601_02527_gb300 as g
    assert torch.cuda.is_available()
    return g


def _overdamped(wl):
    """Q of the first term below 1/2 in every other series (those rows run
    the element pass's second launch, the one with the overdamped branches)."""
    th = wl.theta.copy()
    th[::2, 2] = 0.3
    wl.theta = th
    return wl


def _two_calls(gp, wl, chunk_len):
    m = gp.Model.from_workload(wl, chunk_len=chunk_len)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    ref = m.loglik(th).cpu().numpy()
    n = np.diff(wl.offsets)
    outs = []
    for _ in range(2):
        out = torch.full((wl.n_series,), float("nan"), dtype=torch.float64, device="cuda")
        m.loglik_noalloc(th, out=out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    for got in outs:
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= 1e-4 * np.maximum(np.abs(ref), 0.1 * n))
    return m


@pytest.mark.parametrize("kind", ["sho_m32", "overdamped", "instantaneous"])
def test_noalloc_matches_loglik_two_calls(gp, kind):
    if kind == "sho_m32":
        wl = synth.c2(n_series=24, scale=0.1)
    elif kind == "overdamped":
        wl = _overdamped(synth.c2(n_series=24, scale=0.1))
    else:
        wl = synth.c2i(n_series=24, scale=0.1)
    m = _two_calls(gp, wl, 128)
    if kind == "instantaneous":
        assert m.info["n_slots"] == 0


def _need_bytes(m, n_rows):
    d, nc = m.info["state_dim"], m.info["n_chunks"]
    need = ((2 * d * d + 3 * d) * 4 * nc + 255) // 256 * 256 + 24 * nc
    return need + (800 * 2 * n_rows + 255) // 256 * 256


def test_noalloc_just_under_the_limit(gp):
    # a plan sized to fill most of the fixed array: accepted, same values
    wl = synth.c2(n_series=64, scale=1.0)
    m = gp.Model.from_workload(wl, chunk_len=10)
    need = _need_bytes(m, wl.n_series)
    assert (12 << 20) < need <= (16 << 20), need
    _two_calls(gp, wl, 10)


def test_noalloc_shared_sets(gp):
    wl = synth.c5(n=800, n_sets=3)
    m = gp.Model.from_workload(wl, chunk_len=64)
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    ref = m.loglik(th, per_series=False).cpu().numpy()
    for _ in range(2):
        got = m.loglik_noalloc(th, per_series=False).cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-4 * np.maximum(np.abs(ref), 0.1 * wl.n_meas))


def test_noalloc_rejects_too_large(gp):
    wl = synth.c2(n_series=64, scale=1.5)
    m = gp.Model.from_workload(wl, chunk_len=12)
    assert _need_bytes(m, wl.n_series) > 16 << 20
    th = torch.tensor(wl.theta, dtype=torch.float32, device="cuda")
    with pytest.raises(gp.GPSSError) as e:
        m.loglik_noalloc(th)
    assert e.value.code == 9

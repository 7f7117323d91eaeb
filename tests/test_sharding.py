"""Multi-GPU host logic on CPU ranks: longest-processing-time sharding of
independent series and the gather of per-series rows (gloo, world size 2).
The per-rank compute in this test is the oracle, standing in for each rank's
GPU; what is tested is that the shards cover every series exactly once and
that gathered rows land in global order."""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2601_02527_gb300 import shard


def test_lpt_partition_covers_and_balances():
    rng = np.random.default_rng(3)
    counts = rng.integers(500, 20000, 1024)
    for world in (1, 2, 4, 8):
        parts = shard.lpt_shards(counts, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(counts)))
        loads = [counts[p].sum() for p in parts]
        assert max(loads) - min(loads) <= counts.max()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist

    import oracle
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = synth.c2(n_series=10, scale=0.02)
    parts = shard.lpt_shards(np.diff(wl.offsets), world)
    mine = parts[rank]
    local = oracle.loglik_workload(wl.subset(mine)) if mine else np.zeros(0)
    full = shard.gather_rows(local, mine, wl.n_series)
    if rank == 0:
        np.save(out_path, full)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_gather_matches_unsharded():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp

    import oracle
    import synth
    oracle.build()
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "full.npy")
        tmp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
        got = np.load(out)
    wl = synth.c2(n_series=10, scale=0.02)
    ref = oracle.loglik_workload(wl)
    np.testing.assert_array_equal(got, ref)


# ---------------------------------------------------------------------------
# A single series split in time across ranks.  Each gloo rank forms the
# element of its half of the events with the CUDA path's own chunk-element
# code (elem_event and the element combination, compiled for the host by
# nvcc, run in FP64 with the on-the-fly discretisation), the elements are
# all-gathered by shard.gather_spans -- the exchange the GPU path uses -- and
# folded in time order; the result is the series' log-likelihood, which the
# oracle's sequential filter gives to 1e-9.
# ---------------------------------------------------------------------------
SPAN_SHAPES = {(1, 3): 1, (2, 3): 2}


def _series_for_spans():
    import synth
    wl = synth.c3(n=3000)
    wl.theta = wl.theta.astype(np.float32).astype(np.float64)
    return wl


def _span_rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist

    import paper_2601_02527_gb300 as gp
    from hostmath import harness
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    hh = harness.load()
    wl = _series_for_spans()
    ts, te, y, ye, inst = wl.series(0)
    dt, tag, meas, n_slots = gp.build_events(ts, te, y, ye, inst)
    shape = SPAN_SHAPES[(len(wl.terms), n_slots)]
    nc = hh.hh_span_nc(shape)
    n_ev = len(dt)
    k0, k1 = n_ev * rank // world, n_ev * (rank + 1) // world
    theta = wl.theta[0].astype(np.float32)
    kinds = np.array(list(wl.terms) + [0] * (4 - len(wl.terms)), np.int32)
    elem = np.zeros(nc)
    dt = np.ascontiguousarray(dt)
    tag = np.ascontiguousarray(tag)
    meas = np.ascontiguousarray(meas)
    hh.hh_span_element(shape, dt.ctypes.data, tag.ctypes.data, meas.ctypes.data,
                       theta.ctypes.data, kinds.ctypes.data, k0, k1, 64, elem.ctypes.data)
    allv = shard.gather_spans(torch.from_numpy(elem)[None]).numpy()
    assert allv.shape == (world, 1, nc)
    flat = np.ascontiguousarray(allv[:, 0, :])
    ll = hh.hh_span_fold(shape, flat.ctypes.data, world)
    if rank == 0:
        np.save(out_path, np.array([ll]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_time_split_series_gloo_matches_oracle(world):
    pytest.importorskip("torch")
    import torch.multiprocessing as tmp

    import oracle
    from paper_2601_02527_gb300 import build as gbuild
    gbuild.build()
    oracle.build()
    from hostmath import harness
    harness.load()  # built once, before the ranks start
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "ll.npy")
        tmp.spawn(_span_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        got = float(np.load(out)[0])
    wl = _series_for_spans()
    ref = float(oracle.loglik_workload(wl)[0])
    assert abs(got - ref) <= 1e-9 * abs(ref), (got, ref)


def test_span_chunk_ranges_cover_in_order():
    for n_chunks in (32, 64, 96, 640, 32768, 7):
        for world in (1, 2, 3, 8):
            if n_chunks < world:
                continue
            r = shard.span_chunk_ranges(n_chunks, world)
            assert r[0][0] == 0 and r[-1][1] == n_chunks
            assert all(a < b for a, b in r)
            assert all(r[i][1] == r[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= (32 if n_chunks >= 32 * world else 1)

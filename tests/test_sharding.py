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

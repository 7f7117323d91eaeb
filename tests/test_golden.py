"""The oracle reproduces its stored values (written by tests/golden/make_golden.py)."""
import json
import os

import oracle
import synth

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_c1_golden(oracle_lib):
    with open(os.path.join(HERE, "c1_oracle.json")) as f:
        gold = json.load(f)
    wl = synth.c1()
    ts, te, y, ye, _ = wl.series(0)
    ll, g = oracle.loglik(wl.terms, 0, ts, te, y, ye, wl.theta[0], grad=True)
    assert abs(ll - gold["loglik"]) <= 1e-12 * abs(gold["loglik"])
    assert abs(gold["loglik"] - gold["dense_loglik"]) <= 1e-9 * abs(gold["loglik"])
    for a, b in zip(g, gold["grad"]):
        assert abs(a - b) <= 1e-9 * max(abs(b), 1.0)


def test_f_rows_golden(oracle_lib):
    # overdamped SHO on exposures, instantaneous series, product kernel on
    # instants: the oracle reproduces its stored values, which agree with the
    # dense GP of the same data
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(HERE, "f_oracle.json")) as f:
        gold = json.load(f)
    for name, wl in mg.f_workloads().items():
        ref = gold[name]
        ts, te, y, ye, inst = wl.series(0)
        ll, g = oracle.loglik(wl.terms, wl.layout, ts, te, y, ye, wl.theta[0], instrument=inst,
                              grad=True)
        assert abs(ll - ref["loglik"]) <= 1e-12 * abs(ref["loglik"]), name
        assert abs(ref["loglik"] - ref["dense_loglik"]) <= 1e-9 * abs(ref["loglik"]), name
        for a, b in zip(g, ref["grad"]):
            assert abs(a - b) <= 1e-9 * max(abs(b), 1.0), name

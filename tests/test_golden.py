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

"""Writes the stored expected values under tests/golden/ by calling only oracle/.

The paper prints no numeric worked example (its figures are plots), so the
fixtures here are oracle values on seeded synthetic inputs, kept as a
regression guard for the oracle itself:

  c1_oracle.json  -- the 1000-measurement SHO series (omega0 = 2 pi/10, Q = 3,
                     sigma = 1, s = 0.1), log-likelihood and gradient, plus the
                     dense integrated-GP log-likelihood of the same data.
  f_oracle.json   -- small seeded series of the later rows: an overdamped SHO
                     plus Matern-3/2 on exposures, instantaneous SHO +
                     Matern-3/2 (c2i recipe), and a product kernel plus
                     Matern-3/2 on instants (c2p recipe); log-likelihood,
                     gradient and dense log-likelihood of each.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import dense  # noqa: E402


def main():
    wl = synth.c1()
    ts, te, y, ye, _ = wl.series(0)
    ll, g = oracle.loglik(wl.terms, 0, ts, te, y, ye, wl.theta[0], grad=True)
    ld = dense.loglik(wl.terms, wl.theta[0], ts, te, y, ye)
    out = {"workload": "c1 (synth.c1, seed 1001)", "theta": list(map(float, wl.theta[0])),
           "loglik": ll, "grad": list(map(float, g)), "dense_loglik": ld}
    with open(os.path.join(HERE, "c1_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)
    cases = {}
    for name, wl in f_workloads().items():
        ts, te, y, ye, inst = wl.series(0)
        ll, g = oracle.loglik(wl.terms, wl.layout, ts, te, y, ye, wl.theta[0], instrument=inst,
                              grad=True)
        ld = dense.loglik(wl.terms, wl.theta[0], ts, te, y, ye)
        cases[name] = {"theta": list(map(float, wl.theta[0])), "loglik": ll,
                       "grad": list(map(float, g)), "dense_loglik": ld}
    with open(os.path.join(HERE, "f_oracle.json"), "w") as f:
        json.dump(cases, f, indent=1)
    print(cases)


def f_workloads():
    """The seeded inputs of f_oracle.json (shared with tests/test_golden.py)."""
    import numpy as np
    od = synth.small_single(2001, 150, [1, 2], [1.0, 1.2, 0.2, 0.5, 4.0, 0.1])
    ci = synth.c2i(seed=2002, n_series=1, scale=0.02)
    cp = synth.c2p(seed=2003, n_series=1, scale=0.02)
    for wl in (od, ci, cp):
        wl.theta = np.asarray(wl.theta, np.float64)
    return {"overdamped_exposures": od, "instantaneous": ci, "product_instants": cp}


if __name__ == "__main__":
    main()

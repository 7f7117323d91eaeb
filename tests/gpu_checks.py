"""Checks shared by the GPU parity tests of conditioned values and
predictions (FP32 arithmetic against the FP64 oracle).

A conditioned or predicted variance comes out of the adjoint form as a
prior-sized variance minus the data's reduction of it (h'P*h + 2v'Lv -
(v.l)^2), so its FP32 error scales with the latent's prior variance v0, not
with the (possibly much smaller) result: bound 2e-3 |var| + 2e-4 v0.
Means: 1e-3 max|mean| + 1e-5 |mean|.
"""
import numpy as np

import oracle


def prior_var(terms, layout, theta):
    """The latent's stationary prior variance: the oracle's prediction long
    before a single, uninformative exposure (the series' own data may hold
    coincident resets that the oracle's smoother does not take)."""
    one = np.array([0.0])
    _, v = oracle.predict(terms, layout, one, one + 1.0, one, np.array([1e6]), theta,
                          np.array([-1e4]))
    return float(v[0])


def check_mean_var(got, mean, var, v0):
    gm, gv = got[:, 0].astype(np.float64), got[:, 1].astype(np.float64)
    assert np.all(np.abs(gm - mean) <= 1e-3 * np.abs(mean).max() + 1e-5 * np.abs(mean)), \
        (np.abs(gm - mean).max(), np.abs(mean).max())
    bad = np.abs(gv - var) > 2e-3 * np.abs(var) + 2e-4 * v0
    assert not bad.any(), (np.nonzero(bad)[0][:5], gv[bad][:5], var[bad][:5], v0)

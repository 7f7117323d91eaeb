"""The CUDA path's device arithmetic, built for the host and checked on the CPU.

tests/hostmath/gpss_host_harness.cu compiles the same header functions the
kernels inline (nvcc, host code only).  Checked here:
  * the per-step scalars (f, f', F1, I_ff, I_pp, I_FF) of the table/Horner
    path, the on-the-fly FP32 path and the FP64 path against the oracle's Van
    Loan discretisation over seven decades of step length;
  * their forward-mode derivatives in (a, beta) against central differences
    of the oracle;
  * the economised step-scalar tables against the Taylor series they replace;
  * the pivoted dense solver, the element combination, the closed-form chunk
    log-likelihood and the boundary adjoint against numpy;
  * the observation vector of the update and the conditioned value for
    shapes with and without integral states (instantaneous measurements);
  * the product term's transition and noise (Kronecker of the factors'
    blocks, Eq. product_Q), FP64 and FP32, against the oracle's Van Loan.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def hh():
    from hostmath import harness
    return harness.load()


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def oracle_scalars(w0, q, t):
    """(f, f', F1, I_ff, I_pp, I_FF) from the oracle's Phi~, Q~ (sigma = 1)."""
    Phi, Q, _ = oracle.discretize([1], 0, 1, [1.0, w0, q, 0.1], t)
    qc = 2 * w0 ** 3 / q
    return np.array([Phi[0, 1], Phi[1, 1], Phi[2, 1], Q[0, 0] / qc, Q[1, 1] / qc, Q[2, 2] / qc])


CASES = [(2 * math.pi / 10, 3.0), (math.sqrt(3) / 5, 0.5), (2.0, 0.55), (1.0, 9.5), (8.0, 1.0)]
# overdamped oscillator (Q < 1/2): halving/doubling and two-exponential branches
OVERDAMPED = [(1.0, 0.3), (0.5, 0.05), (2.0, 0.45), (1.0, 0.15), (0.3, 0.499)]


def ab(w0, q):
    return w0 / (2 * q), (w0 * w0 * (1 - 1 / (4 * q * q)) if q != 0.5 else 0.0)


@pytest.mark.parametrize("w0,q", CASES + OVERDAMPED)
def test_step_scalars_match_oracle(oracle_lib, hh, w0, q):
    a, beta = ab(w0, q)
    # up to 40 decay times of the slowest mode (rate ~ omega0 Q for Q << 1/2)
    ts = np.logspace(-5, math.log10(40.0 / min(1.0, 2 * q)), 160) / w0
    refs = np.array([oracle_scalars(w0, q, t) for t in ts])
    floor = np.max(np.abs(refs), axis=0)
    out = np.zeros(6)
    for mode, rtol, ntol in ((0, 6e-6, 3e-7), (1, 6e-6, 3e-7), (2, 1e-11, 1e-13)):
        for t, ref in zip(ts, refs):
            hh.hh_discretize(mode, t, a, beta, _p(out, ctypes.c_double))
            bad = np.abs(out - ref) > rtol * np.abs(ref) + ntol * floor
            assert not bad.any(), (mode, t, w0 * t, out, ref)


@pytest.mark.parametrize("path", ["dual", "tangents"])
@pytest.mark.parametrize("w0,q", [(2 * math.pi / 10, 3.0), (2.0, 0.55), (1.0, 9.5),
                                  (0.7, 0.52), (5.0, 30.0), (1.0, 0.3), (0.5, 0.05), (2.0, 0.45)])
def test_step_scalar_derivatives(oracle_lib, hh, w0, q, path):
    a, beta = ab(w0, q)
    out = np.zeros(18)
    fn = hh.hh_discretize_dual if path == "dual" else hh.hh_discretize_tangents
    xs = (0.01, 0.3, 0.9, 1.1, 1.3, 2.5, 8.0, 30.0)
    if q < 0.5:
        xs = xs + (0.05, 0.15, 90.0, 400.0)
    for x in xs:
        t = x / w0
        fn(t, a, beta, _p(out, ctypes.c_double))
        da, db = out[6:12], out[12:18]
        # chain (a, beta) -> (omega0, Q) and compare with oracle central differences
        g_w0 = da / (2 * q) + db * 2 * w0 * (1 - 1 / (4 * q * q))
        g_q = -da * w0 / (2 * q * q) + db * w0 * w0 / (2 * q ** 3)
        h1, h2 = 1e-6 * w0, 1e-6 * q
        fd_w0 = (oracle_scalars(w0 + h1, q, t) - oracle_scalars(w0 - h1, q, t)) / (2 * h1)
        fd_q = (oracle_scalars(w0, q + h2, t) - oracle_scalars(w0, q - h2, t)) / (2 * h2)
        for got, ref in ((g_w0, fd_w0), (g_q, fd_q)):
            assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-5 * np.max(np.abs(ref))), (x, got, ref)


@pytest.mark.parametrize("w0,q", CASES + OVERDAMPED + [(0.2, 0.55), (9.9, 10.0), (0.05, 30.0),
                                                    (30.0, 0.5), (1.0, 0.02), (1e-3, 3.0),
                                                    (300.0, 3.0)])
def test_table_double_float_path_matches_fp64(hh, w0, q):
    # the table kernel forms the coefficients in double-float arithmetic with
    # the range's scale taken out; against the FP64 construction (same
    # definitions) every coefficient agrees to 1e-12 of its series. size,
    # far inside the FP32 rounding the table is stored with (6e-8)
    a, beta = ab(w0, q)
    assert hh.hh_table_df_check(a, beta) <= 1e-12


@pytest.mark.parametrize("w0,q", CASES + OVERDAMPED + [(0.2, 0.55), (9.9, 10.0), (0.05, 30.0),
                                                    (30.0, 0.5), (1.0, 0.02)])
def test_economised_tables_match_taylor(hh, w0, q):
    # the ten economised coefficients reproduce the 22-term Taylor series on
    # the table's range: the six values to 1e-8 of each series' size (FP32
    # rounding is 6e-8), the twelve (a, beta) tangents, which enter only the
    # gradient, to 1e-6 (worst at critical damping, Q = 1/2: 7e-7)
    a, beta = ab(w0, q)
    assert hh.hh_table_check(a, beta, 0) <= 1e-8
    assert hh.hh_table_check(a, beta, 1) <= 1e-6


@pytest.mark.parametrize("w0,q", CASES + OVERDAMPED)
def test_taylor_generators_agree(hh, w0, q):
    a, beta = ab(w0, q)
    assert hh.hh_taylor_k_check(a, beta) <= 1e-14


@pytest.mark.parametrize("D", [3, 5, 6, 7])
def test_pivoted_solver(hh, D):
    rng = np.random.default_rng(D)
    for trial in range(20):
        A = rng.normal(size=(D, D)).astype(np.float32) + 2 * np.eye(D, dtype=np.float32)
        if trial % 3 == 0:
            A[0, 0] = 0.0  # needs a row exchange
        B = rng.normal(size=(D, 3)).astype(np.float32)
        X = np.zeros((D, 3), np.float32)
        ld = hh.hh_solve(D, _p(A, ctypes.c_float), _p(B, ctypes.c_float), _p(X, ctypes.c_float), 3)
        ref = np.linalg.solve(A.astype(float), B.astype(float))
        assert np.allclose(X, ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
        assert abs(ld - np.linalg.slogdet(A.astype(float))[1]) < 1e-4 * max(1, abs(ld))


def _pk(D, i, j):
    i, j = min(i, j), max(i, j)
    return i * D - i * (i - 1) // 2 + (j - i)


def _pack(S):
    D = S.shape[0]
    return np.array([S[i, j] for i in range(D) for j in range(i, D)], np.float32)


def _unpack(v, D):
    S = np.zeros((D, D))
    for i in range(D):
        for j in range(i, D):
            S[i, j] = S[j, i] = v[_pk(D, i, j)]
    return S


def _rand_elem(rng, D):
    A = rng.normal(size=(D, D)) * 0.5
    b = rng.normal(size=D)
    G = rng.normal(size=(D, D)) * 0.5
    C = G @ G.T
    H = rng.normal(size=(D, D)) * 0.5
    J = H @ H.T
    eta = rng.normal(size=D)
    return A, b, C, eta, J


def _flat(e):
    A, b, C, eta, J = e
    return np.concatenate([A.ravel(), b, _pack(C), eta, _pack(J)]).astype(np.float32)


def _sg21(ei, ej):
    Ai, bi, Ci, ei_, Ji = ei
    Aj, bj, Cj, ej_, Jj = ej
    D = len(bi)
    Mj = Aj @ np.linalg.inv(np.eye(D) + Ci @ Jj)
    Nj = Ai.T @ np.linalg.inv(np.eye(D) + Jj @ Ci)
    return (Mj @ Ai, Mj @ (bi + Ci @ ej_) + bj, Mj @ Ci @ Aj.T + Cj,
            Nj @ (ej_ - Jj @ bi) + ei_, Nj @ Jj @ Ai + Ji)


@pytest.mark.parametrize("shape", [0, 1, 2])
def test_element_combination(hh, shape):
    D = hh.hh_dim(shape)
    rng = np.random.default_rng(10 + shape)
    for _ in range(10):
        ei, ej = _rand_elem(rng, D), _rand_elem(rng, D)
        out = np.zeros(2 * D * D + 3 * D, np.float32)
        hh.hh_combine(shape, _p(_flat(ei), ctypes.c_float), _p(_flat(ej), ctypes.c_float),
                      _p(out, ctypes.c_float))
        ref = _flat(_sg21(ei, ej))
        assert np.allclose(out, ref, rtol=2e-4, atol=2e-4 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [0, 1, 2])
def test_chunk_loglik_and_adjoint(hh, shape):
    D = hh.hh_dim(shape)
    rng = np.random.default_rng(20 + shape)
    for _ in range(10):
        _, _, P, eta, J = _rand_elem(rng, D)
        m = rng.normal(size=D)
        gam, ld, ne = 3.7, -5.2, 11.0
        f32 = lambda a: np.ascontiguousarray(a, np.float32)
        got = hh.hh_chunk_loglik(shape, _p(f32(m), ctypes.c_float), _p(_pack(P), ctypes.c_float),
                                 _p(f32(eta), ctypes.c_float), _p(_pack(J), ctypes.c_float),
                                 gam, ld, ne)
        u = eta - J @ m
        X = np.eye(D) + P @ J
        quad = gam - 2 * eta @ m + m @ J @ m - u @ np.linalg.solve(X, P) @ u
        ref = -0.5 * (ld + ne * math.log(2 * math.pi) + np.linalg.slogdet(X)[1] + quad)
        assert abs(got - ref) <= 1e-4 * max(1.0, abs(ref))
        lam = np.zeros(D, np.float32)
        Lam = np.zeros(D * (D + 1) // 2, np.float32)
        hh.hh_boundary_adjoint(shape, _p(f32(m), ctypes.c_float), _p(_pack(P), ctypes.c_float),
                               _p(f32(eta), ctypes.c_float), _p(_pack(J), ctypes.c_float),
                               _p(lam, ctypes.c_float), _p(Lam, ctypes.c_float))
        Y = np.eye(D) + J @ P
        lref = np.linalg.solve(Y, eta - J @ m)
        Lref = 0.5 * (np.outer(lref, lref) - np.linalg.solve(Y, J))
        assert np.allclose(lam, lref, rtol=1e-4, atol=1e-4 * np.abs(lref).max())
        assert np.allclose(_unpack(Lam, D), Lref, rtol=1e-3, atol=1e-4 * np.abs(Lref).max())


@pytest.mark.parametrize("shape,j,w", [(3, 0, 1.0), (4, 0, 2.5), (4, 1, 0.4), (1, 0, 1.7)])
def test_observation_vector(hh, shape, j, w):
    # the update's h: the latent sum for a shape without integral states
    # (instantaneous measurements), else w on the measurement slot's integral
    # state(s) (one per slot, or one per term under layout 1)
    D = hh.hh_obs_dim(shape)
    h = np.zeros(D)
    if shape == 3:
        h[[0, 2]] = 1.0
    elif shape == 4:
        h[4 + j] = w
    else:
        h[[4, 5]] = w
    rng = np.random.default_rng(30 + shape)
    X = rng.standard_normal((D, D))
    Pm = (X @ X.T + D * np.eye(D)).astype(np.float32)
    Y = rng.standard_normal((D, D))
    Lm = (0.1 * (Y + Y.T)).astype(np.float32)
    m = rng.standard_normal(D).astype(np.float32)
    lam = rng.standard_normal(D).astype(np.float32)
    u = np.zeros(D, np.float32)
    out = np.zeros(4, np.float32)
    hh.hh_observe(shape, j, w, _p(m, ctypes.c_float), _p(Pm, ctypes.c_float),
                  _p(lam, ctypes.c_float), _p(Lm, ctypes.c_float), _p(u, ctypes.c_float),
                  _p(out, ctypes.c_float))
    P64, L64 = Pm.astype(float), Lm.astype(float)
    uref = P64 @ h
    np.testing.assert_allclose(u, uref, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(out[:2], [h @ uref, h @ m], rtol=1e-5, atol=1e-5)
    # conditioned value: smoothed state m + P lam, P - P (lam lam^T - 2 Lam) P
    ms = m + P64 @ lam
    Ps = P64 - P64 @ (np.outer(lam, lam) - 2 * L64) @ P64
    np.testing.assert_allclose(out[2:], [h @ ms, h @ Ps @ h], rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("theta", [(1.3, 0.4, 5.0, 2.1, 0.8), (0.9, 1.1, 0.3, 0.5, 3.0),
                                   (1.0, 2.0, 0.5, 0.7, 0.5)])
def test_product_discretisation(oracle_lib, hh, theta):
    # the kernels' product transition and noise (Kronecker of the factors'
    # blocks, Eq. product_Q) against the oracle's Van Loan of the product model
    th = np.array(list(theta) + [0.1])
    for dt in (0.0, 1e-3, 0.05, 0.7, 3.0, 25.0):
        P_ref, Q_ref, P0 = oracle.discretize([3], 0, 0, th, dt)
        scale = np.abs(P0).max()
        for prec, tol in ((64, 1e-10), (32, 3e-6)):
            Phi = np.zeros(16)
            Q = np.zeros(16)
            hh.hh_prod_disc(prec, dt, _p(th, ctypes.c_double), _p(Phi, ctypes.c_double),
                            _p(Q, ctypes.c_double))
            assert np.all(np.abs(Phi.reshape(4, 4) - P_ref) <= tol * (np.abs(P_ref) + 1)), (prec, dt)
            assert np.all(np.abs(Q.reshape(4, 4) - Q_ref) <= tol * (np.abs(Q_ref) + scale)), (prec, dt)


# (terms, slots, layout) of the harness's covariance-prediction shape ids
_PRED_SHAPES = {0: (1, 1, 0), 1: (1, 3, 0), 2: (2, 1, 1), 3: (2, 3, 0), 4: (2, 2, 0), 5: (2, 0, 0)}


@pytest.mark.parametrize("shape", sorted(_PRED_SHAPES))
def test_covariance_prediction_in_place(hh, shape):
    # the kernels' in-place, one-term-at-a-time P <- Phi P Phi^T + Q against
    # the dense product of the transition and noise the blocks define
    # (Section 3.2: Phi~ maps each term's pair by its 2x2 block; an integral
    # state adds pb0 x + pb1 xdot of the terms it integrates)
    nt, ns, layout = _PRED_SHAPES[shape]
    nz = ns * (1 if layout == 0 or nt == 1 else nt)
    D = 2 * nt + nz
    zs = list(range(2 * nt, D))

    def integrates(z, t):
        return True if (layout == 0 or nt == 1) else (z - 2 * nt) % nt == t

    rng = np.random.default_rng(40 + shape)
    for _ in range(20):
        G = rng.normal(size=(D, D))
        P = G @ G.T
        blk = rng.normal(size=(nt, 12))
        Phi, Q = np.eye(D), np.zeros((D, D))
        for t in range(nt):
            p00, p01, p10, p11, pb0, pb1, q00, q01, q11, qz0, qz1, qzz = blk[t]
            a0, a1 = 2 * t, 2 * t + 1
            Phi[a0, a0], Phi[a0, a1], Phi[a1, a0], Phi[a1, a1] = p00, p01, p10, p11
            Q[a0, a0] += q00
            Q[a0, a1] += q01
            Q[a1, a0] += q01
            Q[a1, a1] += q11
            for z in zs:
                if not integrates(z, t):
                    continue
                Phi[z, a0], Phi[z, a1] = pb0, pb1
                for (i, v) in ((a0, qz0), (a1, qz1)):
                    Q[i, z] += v
                    Q[z, i] += v
                for z2 in zs:
                    if integrates(z2, t):
                        Q[z, z2] += qzz
        ref = Phi @ P @ Phi.T + Q
        v = np.array([P[i, j] for i in range(D) for j in range(i, D)], np.float64)
        b = np.ascontiguousarray(blk.ravel(), np.float64)
        hh.hh_predict_cov(shape, b.ctypes.data, v.ctypes.data)
        np.testing.assert_allclose(_unpack(v, D), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())

"""Parallel-in-time forms of the integrated filter, checked against the oracle.

Section 3.2.5 defers the associative operator to Sarkka & Garcia-Fernandez
(2021): per-event 5-tuples (A, b, C, eta, J) -- an exposure end as in their
Eq. 10, an exposure start as Eq. parallel_ikf_generic, the first event as
Eq. parallel_ikf_first -- combined by their binary operator.  This file
states that operator, and the chunked form used on the GPU, in plain numpy
(FP64) and pins both to the sequential oracle:

* folding the per-event elements left to right, and combining them in a
  balanced tree, both reproduce the oracle's filtered means/covariances and
  log-likelihood;
* a chunk element computed by running the filter from an unknown incoming
  state x (mean M x + b, covariance C, information eta, J about x, plus the
  scalars gamma = sum c^2/S and sum log(2 pi S)) equals the fold of the
  chunk's per-event elements, and its closed-form marginal log-likelihood
  given N(m, P) for x equals the oracle's sum over the chunk;
* the derivative of the log-likelihood of all later data with respect to the
  filtered state (m, P) at a chunk boundary is lambda = (I + J P)^-1 (eta - J m)
  and Lambda = (lambda lambda^T - (I + J P)^-1 J) / 2 (checked by central
  differences), the quantity the reverse-time gradient starts from.
"""
import math

import numpy as np
import pytest

import oracle
import synth

SHO, M32 = 1, 2


def zidx(terms, layout, slot):
    T = len(terms)
    if layout == 0:
        return [2 * T + slot]
    return [2 * T + slot * T + t for t in range(T)]


def event_mats(terms, layout, ts, te, y, ye, theta, inst=None):
    ev = oracle.events(ts, te, y, ye, inst)
    S = ev["n_slots"]
    D = oracle.dim(terms, layout, S)
    s2 = theta[-1] ** 2
    out = []
    tprev = ev["t"][0]
    for k in range(len(ev["t"])):
        dt = ev["t"][k] - tprev
        tprev = ev["t"][k]
        Phi, Q, P0 = oracle.discretize(terms, layout, S, theta, dt)
        z = zidx(terms, layout, ev["slot"][k])
        if ev["kind"][k] == 0:
            R = np.eye(D)
            for i in z:
                R[i, i] = 0
            out.append(dict(kind=0, Phi=Phi, Q=Q, R=R))
        else:
            h = np.zeros(D)
            h[z] = ev["invd"][k]
            out.append(dict(kind=1, Phi=Phi, Q=Q, h=h, r=ev["r0"][k] + s2, y=ev["y"][k]))
    return out, P0, D


def sequential(evm, P0, D, m0=None, start=0):
    m = np.zeros(D) if m0 is None else m0.copy()
    P = P0.copy()
    ll = 0.0
    states = []
    for e in evm[start:]:
        m = e["Phi"] @ m
        P = e["Phi"] @ P @ e["Phi"].T + e["Q"]
        if e["kind"] == 0:
            m = e["R"] @ m
            P = e["R"] @ P @ e["R"]
        else:
            h = e["h"]
            S = h @ P @ h + e["r"]
            v = e["y"] - h @ m
            K = P @ h / S
            m = m + K * v
            P = P - np.outer(K, K) * S
            ll += -0.5 * (math.log(2 * math.pi * S) + v * v / S)
        P = 0.5 * (P + P.T)
        states.append((m.copy(), P.copy()))
    return ll, states


def element(e, first=False, P0=None):
    D = e["Phi"].shape[0]
    A, Q = e["Phi"], e["Q"]
    if first:
        # G11 reading: A_1 = 0, b_1 and C_1 the reset predicted prior
        R = e["R"]
        return (np.zeros((D, D)), np.zeros(D), R @ (A @ P0 @ A.T + Q) @ R, np.zeros(D),
                np.zeros((D, D)))
    if e["kind"] == 0:
        R = e["R"]
        return (R @ A, np.zeros(D), R @ Q @ R, np.zeros(D), np.zeros((D, D)))
    h, r, y = e["h"], e["r"], e["y"]
    S = h @ Q @ h + r
    K = Q @ h / S
    IKh = np.eye(D) - np.outer(K, h)
    return (IKh @ A, K * y, IKh @ Q, A.T @ h * y / S, np.outer(A.T @ h, A.T @ h) / S)


def combine(ei, ej):
    Ai, bi, Ci, ei_, Ji = ei
    Aj, bj, Cj, ej_, Jj = ej
    D = len(bi)
    Mj = Aj @ np.linalg.inv(np.eye(D) + Ci @ Jj)
    Nj = Ai.T @ np.linalg.inv(np.eye(D) + Jj @ Ci)
    return (Mj @ Ai, Mj @ (bi + Ci @ ej_) + bj, Mj @ Ci @ Aj.T + Cj,
            Nj @ (ej_ - Jj @ bi) + ei_, Nj @ Jj @ Ai + Ji)


def tree_scan(elems):
    """Inclusive prefix by recursive doubling (Hillis-Steele)."""
    cur = list(elems)
    step = 1
    while step < len(cur):
        nxt = list(cur)
        for i in range(step, len(cur)):
            nxt[i] = combine(cur[i - step], cur[i])
        cur = nxt
        step *= 2
    return cur


def chunk_element(evm, a, b, D, m_known=None, P_known=None):
    """Run the filter over events a..b-1 from an unknown x (or a known state)."""
    if m_known is None:
        Mx, bb, C = np.eye(D), np.zeros(D), np.zeros((D, D))
    else:
        Mx, bb, C = np.zeros((D, D)), m_known.copy(), P_known.copy()
    eta, J, gam, ld = np.zeros(D), np.zeros((D, D)), 0.0, 0.0
    for e in evm[a:b]:
        Mx, bb = e["Phi"] @ Mx, e["Phi"] @ bb
        C = e["Phi"] @ C @ e["Phi"].T + e["Q"]
        if e["kind"] == 0:
            Mx, bb, C = e["R"] @ Mx, e["R"] @ bb, e["R"] @ C @ e["R"]
        else:
            h = e["h"]
            u = C @ h
            S = h @ u + e["r"]
            c = e["y"] - h @ bb
            g = h @ Mx
            J = J + np.outer(g, g) / S
            eta = eta + g * c / S
            gam += c * c / S
            ld += math.log(2 * math.pi * S)
            K = u / S
            Mx = Mx - np.outer(K, g)
            bb = bb + K * c
            C = C - np.outer(u, u) / S
        C = 0.5 * (C + C.T)
    return dict(A=Mx, b=bb, C=C, eta=eta, J=J, gam=gam, ld=ld)


def chunk_loglik(el, m, P):
    D = len(m)
    eta, J = el["eta"], el["J"]
    u = eta - J @ m
    IPJ = np.eye(D) + P @ J
    W = np.linalg.solve(IPJ, P)
    quad = el["gam"] - 2 * eta @ m + m @ J @ m - u @ W @ u
    return -0.5 * (el["ld"] + np.linalg.slogdet(IPJ)[1] + quad)


def _case(kind):
    if kind == "single":
        wl = synth.small_single(51, 40, [SHO, M32], [1.0, 0.9, 3.0, 0.5, 4.0, 0.1])
        return wl.terms, 0, wl.series(0), wl.theta[0]
    if kind == "layout1":
        wl = synth.small_single(52, 35, [SHO, SHO], [1.0, 0.7, 3.0, 0.5, 3.0, 1.2, 0.1])
        return wl.terms, 1, wl.series(0), wl.theta[0]
    wl = synth.two_instrument_overlap(53, 30, 12)
    return wl.terms, 0, wl.series(0), wl.theta[0]


@pytest.mark.parametrize("kind", ["single", "layout1", "overlap"])
def test_sg21_elements_reproduce_oracle(oracle_lib, kind):
    terms, layout, (ts, te, y, ye, inst), theta = _case(kind)
    evm, P0, D = event_mats(terms, layout, ts, te, y, ye, theta, inst)
    ll_seq, states = sequential(evm, P0, D)
    ll_or = oracle.loglik(terms, layout, ts, te, y, ye, theta, instrument=inst)
    assert abs(ll_seq - ll_or) <= 1e-11 * abs(ll_or)
    elems = [element(evm[0], first=True, P0=P0)] + [element(e) for e in evm[1:]]
    fold = [elems[0]]
    for e in elems[1:]:
        fold.append(combine(fold[-1], e))
    tree = tree_scan(elems)
    for k, (m, P) in enumerate(states):
        for pre in (fold[k], tree[k]):
            np.testing.assert_allclose(pre[1], m, rtol=1e-9, atol=1e-11)
            np.testing.assert_allclose(pre[2], P, rtol=1e-9, atol=1e-11)
    # log-likelihood from the prefix states: predict one step from k-1
    ll = 0.0
    for k, e in enumerate(evm):
        if e["kind"] == 1:
            m, P = tree[k - 1][1], tree[k - 1][2]
            mp_, Pp = e["Phi"] @ m, e["Phi"] @ P @ e["Phi"].T + e["Q"]
            S = e["h"] @ Pp @ e["h"] + e["r"]
            v = e["y"] - e["h"] @ mp_
            ll += -0.5 * (math.log(2 * math.pi * S) + v * v / S)
    assert abs(ll - ll_or) <= 1e-9 * abs(ll_or)


@pytest.mark.parametrize("kind", ["single", "layout1", "overlap"])
@pytest.mark.parametrize("L", [5, 16])
def test_chunk_elements_and_closed_form_loglik(oracle_lib, kind, L):
    terms, layout, (ts, te, y, ye, inst), theta = _case(kind)
    evm, P0, D = event_mats(terms, layout, ts, te, y, ye, theta, inst)
    ll_or = oracle.loglik(terms, layout, ts, te, y, ye, theta, instrument=inst)
    _, states = sequential(evm, P0, D)
    K = len(evm)
    bounds = list(range(0, K, L)) + [K]
    total = 0.0
    m_in, P_in = None, None
    for c in range(len(bounds) - 1):
        a, b = bounds[c], bounds[c + 1]
        if c == 0:
            el = chunk_element(evm, a, b, D, np.zeros(D), P0)
            assert np.all(el["A"] == 0) and np.all(el["J"] == 0)
            total += -0.5 * (el["ld"] + el["gam"])
        else:
            el = chunk_element(evm, a, b, D)
            # the chunk element equals the fold of its per-event elements
            f = element(evm[a])
            for e in evm[a + 1:b]:
                f = combine(f, element(e))
            for got, ref in zip((el["A"], el["b"], el["C"], el["eta"], el["J"]), f):
                np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-10)
            total += chunk_loglik(el, m_in, P_in)
            # state-combine: filtered state at the chunk end
            IPJ = np.eye(D) + P_in @ el["J"]
            m_out = el["A"] @ np.linalg.solve(IPJ, m_in + P_in @ el["eta"]) + el["b"]
            P_out = el["A"] @ np.linalg.solve(IPJ, P_in) @ el["A"].T + el["C"]
            np.testing.assert_allclose(m_out, states[b - 1][0], rtol=1e-8, atol=1e-10)
            np.testing.assert_allclose(P_out, states[b - 1][1], rtol=1e-8, atol=1e-10)
        m_in, P_in = states[b - 1]
    assert abs(total - ll_or) <= 1e-9 * abs(ll_or)


def test_boundary_adjoint_formula(oracle_lib):
    terms, layout, (ts, te, y, ye, inst), theta = _case("overlap")
    evm, P0, D = event_mats(terms, layout, ts, te, y, ye, theta, inst)
    _, states = sequential(evm, P0, D)
    kb = 41  # boundary after event kb
    m, P = states[kb]
    el = chunk_element(evm, kb + 1, len(evm), D)
    J, eta = el["J"], el["eta"]
    IJP = np.eye(D) + J @ P
    lam = np.linalg.solve(IJP, eta - J @ m)
    Lam = 0.5 * (np.outer(lam, lam) - np.linalg.solve(IJP, J))

    def rest(mm, PP):
        # filter from (mm, PP) over the remaining events
        evr = evm[kb + 1:]
        ll, _ = sequential(evr, PP, D, m0=mm)
        return ll

    h = 1e-6
    for i in range(D):
        dm = np.zeros(D)
        dm[i] = h
        fd = (rest(m + dm, P) - rest(m - dm, P)) / (2 * h)
        assert abs(fd - lam[i]) <= 1e-6 * max(1.0, abs(lam[i]))
    for i in range(D):
        for j in range(i, D):
            E = np.zeros((D, D))
            E[i, j] = E[j, i] = h
            fd = (rest(m, P + E) - rest(m, P - E)) / (2 * h)
            ref = Lam[i, j] if i == j else 2 * Lam[i, j]
            assert abs(fd - ref) <= 1e-5 * max(1.0, abs(ref)), (i, j, fd, ref)

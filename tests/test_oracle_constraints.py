"""Pins of the oracle's constraint rows (the paragraph on state/input
constraints after Table I of arXiv 2410.09663): a constraint g(X, U) <= 0 is
observed as z = phi(g) + eps with reference 0, phi(x) = ln(1 + e^{beta x}) /
alpha, and z joins the pseudo-observation Ybar_t of every assimilation time.

The pins do not retype the oracle's formulas: the barrier against closed
forms and limits, the constraint rows against a hand-worked case, the solve
against a rebuild from pieces pinned elsewhere (CNN step, textbook analysis),
and a solve whose control reference lies outside a box against the
barrier's intended effect."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_09663_b300 import workloads


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (10.0, 100.0), (0.5, 3.0)])
def test_softplus_barrier_closed_forms(alpha, beta):
    phi = lambda x: oracle.softplus_barrier(x, alpha, beta)
    assert phi(0.0) == pytest.approx(math.log(2.0) / alpha, rel=1e-15)
    # ln(1 + (e - 1)) = 1
    assert phi(math.log(math.e - 1.0) / beta) == pytest.approx(1.0 / alpha, rel=1e-14)
    # softplus(y) - softplus(-y) = y
    for x in (0.013, 0.4, 2.5, 7.0):
        assert phi(x) - phi(-x) == pytest.approx(beta * x / alpha, rel=1e-12)


def test_softplus_barrier_limits():
    alpha, beta = 10.0, 100.0
    # far inside the feasible set the barrier vanishes like e^{beta x} / alpha
    x = -0.3
    assert oracle.softplus_barrier(x, alpha, beta) == pytest.approx(math.exp(beta * x) / alpha, rel=1e-12)
    # far outside it grows like beta x / alpha, and e^{beta x} never overflows
    for x in (0.5, 20.0, 1e3):
        assert oracle.softplus_barrier(x, alpha, beta) == pytest.approx(beta * x / alpha, rel=1e-15)
    assert oracle.softplus_barrier(-1e3, alpha, beta) == 0.0


def test_constraint_obs_hand_worked():
    # n = 2, l = 1, m = 2, two constraint rows
    X = np.array([[1.0, 2.0], [3.0, 4.0]])
    U = np.array([[0.5, -1.0]])
    cons = oracle.Cons(Gx=[[1.0, 0.0], [0.0, -1.0]], Gu=[[2.0], [0.0]], h=[0.5, -3.0], alpha=2.0, beta=1.0)
    # row 0: X[0] + 2 U[0] - 0.5 = [1.5, -0.5];  row 1: -X[1] + 3 = [0, -1]
    g = np.array([[1.5, -0.5], [0.0, -1.0]])
    eps = np.array([[0.01, -0.02], [0.03, 0.0]])
    z = oracle.constraint_obs(cons, X, U, eps)
    want = np.array([[oracle.softplus_barrier(v, 2.0, 1.0) for v in row] for row in g]) + eps
    np.testing.assert_allclose(z, want, rtol=0, atol=1e-15)
    assert z[1, 0] == pytest.approx(math.log(2.0) / 2.0 + 0.03, rel=1e-15)


def _tiny_net(rng, n, m, l):
    C = 3
    w1 = 0.3 * rng.standard_normal((C, 2, 3, 3))
    w2 = 0.3 * rng.standard_normal((1, C, 3, 3))
    b1 = 0.1 * rng.standard_normal(C)
    b2 = 0.1 * rng.standard_normal(1)
    B = rng.standard_normal((n, l))
    return oracle.Net(n, m, l, [2, C, 1], [(w1, b1), (w2, b2)], B, residual_scale=0.1)


def test_constrained_solve_h1_rebuilt_from_pinned_pieces():
    """One assimilation (H = 1): ensemble init, one prediction, the constraint
    rows at the predicted X_1, U_1 with reference 0, the analysis on the
    full history; rebuilt here from oracle.cnn_step, oracle.constraint_obs and
    oracle.enks_analysis, each pinned on its own."""
    rng = np.random.default_rng(71)
    n, m, l, N, H, c = 4, 4, 2, 24, 1, 3
    net = _tiny_net(rng, n, m, l)
    cons = oracle.Cons(Gx=rng.standard_normal((c, n)), Gu=rng.standard_normal((c, l)),
                       h=rng.standard_normal(c), alpha=2.0, beta=3.0)
    X_k = rng.standard_normal((n, m))
    U_prev = 0.1 * rng.standard_normal((l, m))
    X_ref = rng.standard_normal((H + 1, n, m))
    U_ref = 0.1 * rng.standard_normal((l, m))
    W0 = 0.1 * rng.standard_normal((N, l, m))
    W = 0.1 * rng.standard_normal((H, N, l, m))
    VX = 0.1 * rng.standard_normal((H, N, n, m))
    VU = 0.1 * rng.standard_normal((H, N, l, m))
    VZ = 0.1 * rng.standard_normal((H, N, c, m))
    noise = np.concatenate([a.ravel() for a in (W0, W, VX, VU, VZ)])
    got = oracle.enks_solve(net, N, H, X_k, U_prev, X_ref, U_ref, noise, cons)

    q = n + 2 * l
    hist = np.zeros((N, 2 * q, m))
    Y = np.zeros((N, n + l + c, m))
    for i in range(N):
        U0 = U_prev + W0[i]
        X1 = oracle.cnn_step(net, X_k, U0)
        U1 = U0 + W[0, i]
        hist[i, :n], hist[i, n:n + l], hist[i, n + l:q] = X_k, U0, W0[i]
        hist[i, q:q + n], hist[i, q + n:q + n + l], hist[i, q + n + l:] = X1, U1, W[0, i]
        Y[i, :n] = X1 + VX[0, i]
        Y[i, n:n + l] = U1 + VU[0, i]
        Y[i, n + l:] = oracle.constraint_obs(cons, X1, U1, VZ[0, i])
    Ybar = np.concatenate([X_ref[1], U_ref, np.zeros((c, m))])
    post = oracle.enks_analysis(hist, Y, Ybar).mean(0)
    np.testing.assert_allclose(got.reshape(2 * q, m), post, rtol=0, atol=1e-12)

    # and the constraint rows matter: without them the result differs
    plain = oracle.enks_solve(net, N, H, X_k, U_prev, X_ref, U_ref, noise[:noise.size - VZ.size])
    assert np.abs(plain - got).max() > 1e-6


def test_constraint_noise_leaves_the_other_noise_unchanged():
    wl = workloads.small_16()
    wc = wl.with_(cons=workloads.u_box(wl.n, wl.l, 0.1))
    a, b = wl.noise(3), wc.noise(3)
    assert b.size == a.size + wl.H * wl.N * 2 * wl.l * wl.m == wc.noise_floats()
    np.testing.assert_array_equal(b[:a.size], a)


def _violation(U, u_max):
    return float(np.maximum(np.abs(U) - u_max, 0.0).sum())


@pytest.mark.parametrize("k", [0, 1])
def test_box_constraint_pulls_the_plan_to_the_bound(k):
    """Algorithm 1 assimilates at t = k+1 .. k+H, so the barrier acts on the
    planned controls U_{k+1} .. U_{k+H} (not directly on the applied U_k).
    With U^ref = 0.2 outside the box |U| <= 0.1 the unconstrained plan follows
    the reference; with the barrier rows it sits at the bound: the sign and the
    strength of the barrier's pull."""
    wl = workloads.small_16()
    u_max = 0.1
    wc = wl.with_(cons=workloads.u_box(wl.n, wl.l, u_max))
    net = oracle.Net(wl.n, wl.m, wl.l, wl.channels, wl.weights(), wl.B(), wl.residual_scale)
    cw = wc.cons
    cons = oracle.Cons(cw.Gx, cw.Gu, cw.h, cw.alpha, cw.beta)
    X_ref = wl.X_ref_all(4)[k:k + wl.H + 1]
    U_ref = np.full((wl.l, wl.m), 0.2)
    U_prev = np.zeros((wl.l, wl.m))
    a = oracle.enks_solve(net, wl.N, wl.H, wl.X0(), U_prev, X_ref, U_ref, wl.noise(k))
    b = oracle.enks_solve(net, wl.N, wl.H, wl.X0(), U_prev, X_ref, U_ref, wc.noise(k), cons)
    ua = a[1:, wl.n:wl.n + wl.l]
    ub = b[1:, wl.n:wl.n + wl.l]
    assert ua.mean() > 0.17                          # follows U^ref without the barrier
    assert abs(ub.mean() - u_max) < 0.02             # held at the bound with it
    assert _violation(ub, u_max) < 0.25 * _violation(ua, u_max)

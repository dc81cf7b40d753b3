"""Pins of the oracle's optional covariance outputs (Algorithm 1's steps that
the paper lets be skipped): the ensemble row covariance of Eq.
(ensemble-based-Kalman-update-cov) and Eq. (prediction-cov) .. Eq.
(prediction-cov-concatenate), taken after every prediction and every update.

The row covariance is pinned against numpy's per-column covariance, the solve
against a rebuild from pinned pieces, and the pair (prior, posterior) against
the exact identity of the perturbed-observation update,
    S(A') = S(A) - S(A, B) S(B)^{-1} S(B, A),   A' = A - K B,  K = S(A, B) S(B)^{-1},
which also fixes the sign of the covariance update (the Appendix's "-")."""
import numpy as np
import pytest

import oracle


def test_row_cov_matches_numpy_per_column():
    rng = np.random.default_rng(81)
    N, R, m = 17, 6, 5
    X = rng.standard_normal((N, R, m)) + rng.standard_normal((1, R, m))
    want = sum(np.cov(X[:, :, j].T, bias=True) for j in range(m))
    np.testing.assert_allclose(oracle.row_cov(X), want, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(oracle.row_cov(X, lam=0.3), 0.3 * want, rtol=1e-12, atol=1e-13)


def _tiny(rng, n, m, l):
    C = 3
    w1 = 0.3 * rng.standard_normal((C, 2, 3, 3))
    w2 = 0.3 * rng.standard_normal((1, C, 3, 3))
    B = rng.standard_normal((n, l))
    return oracle.Net(n, m, l, [2, C, 1], [(w1, 0.1 * rng.standard_normal(C)), (w2, 0.1 * rng.standard_normal(1))],
                      B, residual_scale=0.1)


def _inputs(rng, n, m, l, N, H):
    X_k = rng.standard_normal((n, m))
    U_prev = 0.1 * rng.standard_normal((l, m))
    X_ref = rng.standard_normal((H + 1, n, m))
    U_ref = 0.1 * rng.standard_normal((l, m))
    parts = [0.1 * rng.standard_normal(s) for s in ((N, l, m), (H, N, l, m), (H, N, n, m), (H, N, l, m))]
    return X_k, U_prev, X_ref, U_ref, parts


def test_solve_cov_h1_rebuilt_and_posterior_identity():
    rng = np.random.default_rng(82)
    n, m, l, N, H = 4, 5, 2, 30, 1
    net = _tiny(rng, n, m, l)
    X_k, U_prev, X_ref, U_ref, (W0, W, VX, VU) = _inputs(rng, n, m, l, N, H)
    noise = np.concatenate([a.ravel() for a in (W0, W, VX, VU)])
    xh, pred, post = oracle.enks_solve_cov(net, N, H, X_k, U_prev, X_ref, U_ref, noise)
    np.testing.assert_array_equal(xh, oracle.enks_solve(net, N, H, X_k, U_prev, X_ref, U_ref, noise))

    q = n + 2 * l
    hist = np.zeros((N, 2 * q, m))
    Y = np.zeros((N, n + l, m))
    for i in range(N):
        U0 = U_prev + W0[i]
        X1 = oracle.cnn_step(net, X_k, U0)
        U1 = U0 + W[0, i]
        hist[i] = np.concatenate([X_k, U0, W0[i], X1, U1, W[0, i]])
        Y[i] = np.concatenate([X1 + VX[0, i], U1 + VU[0, i]])
    np.testing.assert_allclose(pred[0], oracle.row_cov(hist), rtol=0, atol=1e-13)
    after = oracle.enks_analysis(hist, Y, np.concatenate([X_ref[1], U_ref]))
    np.testing.assert_allclose(post[0], oracle.row_cov(after), rtol=0, atol=1e-13)

    # exact identity of the update: S(A') = S(A) - S_XY S_Y^{-1} S_YX (moments
    # with 1/N, the same normalisation as row_cov with lambda = 1)
    _, _, cxy, cyy = oracle.moments(hist, Y)
    np.testing.assert_allclose(cyy, oracle.row_cov(Y), rtol=1e-12)      # same 1/N normalisation
    ident = pred[0] - cxy @ np.linalg.solve(cyy, cxy.T)
    np.testing.assert_allclose(post[0], ident, rtol=0, atol=1e-12)
    # the update shrinks the spread: the identity's correction is positive semidefinite
    assert np.trace(post[0]) < np.trace(pred[0])


@pytest.mark.parametrize("lam", [0.25, 3.0])
def test_solve_cov_lambda_scales_both_outputs(lam):
    rng = np.random.default_rng(83)
    n, m, l, N, H = 3, 4, 1, 20, 2
    net = _tiny(rng, n, m, l)
    X_k, U_prev, X_ref, U_ref, parts = _inputs(rng, n, m, l, N, H)
    noise = np.concatenate([a.ravel() for a in parts])
    _, p1, q1 = oracle.enks_solve_cov(net, N, H, X_k, U_prev, X_ref, U_ref, noise)
    _, pl, ql = oracle.enks_solve_cov(net, N, H, X_k, U_prev, X_ref, U_ref, noise, lam=lam)
    for s in range(H):
        np.testing.assert_allclose(pl[s], lam * p1[s], rtol=1e-14, atol=0)
        np.testing.assert_allclose(ql[s], lam * q1[s], rtol=1e-14, atol=0)
        # the prediction to t = k+s+1 extends the previous posterior: its
        # leading blocks are the previous update's covariance
        if s > 0:
            r = q1[s - 1].shape[0]
            np.testing.assert_allclose(p1[s][:r, :r], q1[s - 1], rtol=0, atol=1e-14)

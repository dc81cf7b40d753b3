"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Every test here runs on the CPU.  None of them retypes the oracle's formula:
each compares it with a library routine used differently, a closed form, a
hand-derived case, an invariant, or an independent textbook algorithm.
"""
import json
import os

import numpy as np
import pytest
from scipy import signal

import oracle
from paper_2410_09663_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- P1: conv
def _im2col_conv(x, w, b):
    """Independent formulation: zero-pad, gather the nine shifted planes and
    contract with a matrix product."""
    cin, n, m = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    cols = np.stack([xp[:, dy:dy + n, dx:dx + m] for dy in range(3) for dx in range(3)], axis=1)
    cols = cols.reshape(cin * 9, n * m)                      # (c, dy, dx) x pixels
    return (w.reshape(w.shape[0], cin * 9) @ cols).reshape(-1, n, m) + b[:, None, None]


def test_conv_matches_im2col_matmul():
    rng = np.random.default_rng(11)
    for (cin, cout, n, m) in [(3, 4, 7, 9), (1, 1, 1, 1), (2, 5, 1, 6), (4, 2, 5, 1)]:
        x = rng.standard_normal((cin, n, m))
        w = rng.standard_normal((cout, cin, 3, 3))
        b = rng.standard_normal(cout)
        got = oracle.conv3x3(x, w, b)
        np.testing.assert_allclose(got, _im2col_conv(x, w, b), rtol=0, atol=1e-12)
        np.testing.assert_allclose(oracle.conv3x3(x, w, b, apply_tanh=True),
                                   np.tanh(_im2col_conv(x, w, b)), rtol=0, atol=1e-12)


def test_conv_matches_scipy_correlate2d():
    rng = np.random.default_rng(12)
    x = rng.standard_normal((1, 13, 10))
    w = rng.standard_normal((1, 1, 3, 3))
    want = signal.correlate2d(x[0], w[0, 0], mode="same", boundary="fill", fillvalue=0.0)
    np.testing.assert_allclose(oracle.conv3x3(x, w, np.zeros(1))[0], want, atol=1e-12)


def test_conv_discrete_laplacian_of_quadratic_is_constant():
    # f = a y^2 + b x^2 + c x y + d y + e x + g has 5-point Laplacian 2a + 2b.
    n, m = 9, 11
    y, x = np.mgrid[0:n, 0:m].astype(float)
    a, b, c, d, e, g = 0.7, -0.3, 0.25, 1.5, -2.0, 0.125
    f = a * y * y + b * x * x + c * x * y + d * y + e * x + g
    L = np.array([[0, 1, 0], [1, -4, 1], [0, 1, 0]], float)[None, None]
    out = oracle.conv3x3(f[None], L, np.zeros(1))[0]
    np.testing.assert_allclose(out[1:-1, 1:-1], 2 * a + 2 * b, atol=1e-10)


def test_cnn_step_single_linear_layer_closed_form():
    # One linear layer 2 -> 1 with only centre taps: X' = X + s (w0 X + w1 B U + b).
    rng = np.random.default_rng(13)
    n, m, l = 5, 7, 3
    w = np.zeros((1, 2, 3, 3))
    w[0, 0, 1, 1], w[0, 1, 1, 1] = 0.6, -1.3
    bias = np.array([0.2])
    B = rng.standard_normal((n, l))
    net = oracle.Net(n, m, l, [2, 1], [(w, bias)], B, residual_scale=0.1)
    X, U = rng.standard_normal((n, m)), rng.standard_normal((l, m))
    want = X + 0.1 * (0.6 * X - 1.3 * (B @ U) + 0.2)
    np.testing.assert_allclose(oracle.cnn_step(net, X, U), want, atol=1e-12)


def test_cnn_step_hidden_tanh_closed_form():
    # Hidden layer with only biases active gives tanh(b1) everywhere; the last
    # layer's centre tap then adds w2 * tanh(b1) + b2 (plus edge effects of the
    # off-centre taps, which are zero here).
    n, m, l = 4, 6, 2
    w1 = np.zeros((3, 2, 3, 3))
    b1 = np.array([0.5, -1.0, 2.0])
    w2 = np.zeros((1, 3, 3, 3))
    w2[0, :, 1, 1] = [1.0, 2.0, -0.5]
    b2 = np.array([0.3])
    net = oracle.Net(n, m, l, [2, 3, 1], [(w1, b1), (w2, b2)], np.ones((n, l)))
    X = np.full((n, m), 0.25)
    out = oracle.cnn_step(net, X, np.ones((l, m)))
    want = 0.25 + 0.1 * (np.tanh(0.5) + 2 * np.tanh(-1.0) - 0.5 * np.tanh(2.0) + 0.3)
    np.testing.assert_allclose(out, want, atol=1e-12)


def test_cnn_step_batch_equals_single():
    wl = W.small_16()
    net = oracle.Net(wl.n, wl.m, wl.l, wl.channels, wl.weights(), wl.B())
    rng = np.random.default_rng(3)
    X = rng.standard_normal((5, wl.n, wl.m))
    U = rng.standard_normal((5, wl.l, wl.m))
    got = oracle.cnn_step(net, X, U)
    for i in range(5):
        np.testing.assert_array_equal(got[i], oracle.cnn_step(net, X[i], U[i]))


# --------------------------------------------------- P2: means, covariances
def test_golden_two_member_updates():
    cases = json.load(open(os.path.join(GOLDEN, "two_member_update.json")))["cases"]
    for c in cases:
        X = np.array(c["X"], float)
        V = np.array(c["V"], float)
        Y = X[:, c["obs_rows"], :] + V
        xm, ym, cxy, cyy = oracle.moments(X, Y)
        np.testing.assert_allclose(cxy, c["Cxy"], atol=1e-14)
        np.testing.assert_allclose(cyy, c["Cyy"], atol=1e-14)
        np.testing.assert_allclose(oracle.gain(cxy, cyy), c["K"], atol=1e-14)
        np.testing.assert_allclose(oracle.enks_analysis(X, Y, np.array(c["Ybar"])), c["X_post"],
                                   atol=1e-13)


def test_moments_two_members_hand_formula():
    # With two members the anomalies are +-d/2, so (1/N) sum_i a_i b_i^T = d_a d_b^T / 4
    # summed over columns.
    rng = np.random.default_rng(21)
    X = rng.standard_normal((2, 4, 5))
    Y = rng.standard_normal((2, 3, 5))
    _, _, cxy, cyy = oracle.moments(X, Y)
    dx, dy = X[0] - X[1], Y[0] - Y[1]
    np.testing.assert_allclose(cxy, dx @ dy.T / 4, atol=1e-13)
    np.testing.assert_allclose(cyy, dy @ dy.T / 4, atol=1e-13)


def test_moments_match_numpy_cov_per_column():
    rng = np.random.default_rng(22)
    N, R, p, m = 9, 4, 3, 6
    X = rng.standard_normal((N, R, m))
    Y = rng.standard_normal((N, p, m))
    xm, ym, cxy, cyy = oracle.moments(X, Y)
    np.testing.assert_allclose(xm, X.mean(0), atol=1e-14)
    np.testing.assert_allclose(ym, Y.mean(0), atol=1e-14)
    cxy_ref = sum(np.cov(X[:, :, j].T, Y[:, :, j].T, bias=True)[:R, R:] for j in range(m))
    cyy_ref = sum(np.cov(Y[:, :, j].T, bias=True) for j in range(m))
    np.testing.assert_allclose(cxy, cxy_ref, atol=1e-12)
    np.testing.assert_allclose(cyy, cyy_ref, atol=1e-12)


def test_moments_member_permutation_invariant():
    rng = np.random.default_rng(23)
    X = rng.standard_normal((7, 5, 4))
    Y = rng.standard_normal((7, 3, 4))
    perm = rng.permutation(7)
    a = oracle.moments(X, Y)
    b = oracle.moments(X[perm], Y[perm])
    for u, v in zip(a, b):
        np.testing.assert_allclose(u, v, atol=1e-13)


def test_matrix_normal_row_covariance_moment():
    # Appendix: X ~ MN(M; Sigma, Psi) has E[(X-M)(X-M)^T] = tr(Psi) Sigma.
    # The oracle's row covariance must estimate tr(Psi) Sigma (not tr(Sigma) Psi,
    # which a transposed operand would give).
    rng = np.random.default_rng(24)
    n, m, N = 3, 4, 200000
    A = np.array([[1.0, 0, 0], [0.5, 1.0, 0], [-0.3, 0.2, 0.7]])
    Bm = np.array([[1.0, 0, 0, 0], [0.3, 0.5, 0, 0], [0, 0.2, 1.2, 0], [0.1, 0, 0.4, 0.3]])
    Sigma, Psi = A @ A.T, Bm @ Bm.T
    Z = rng.standard_normal((N, n, m))
    X = A[None] @ Z @ Bm.T[None]
    _, _, _, cyy = oracle.moments(X, X)
    np.testing.assert_allclose(cyy, np.trace(Psi) * Sigma, atol=0.03 * np.trace(Psi) * np.abs(Sigma).max())
    # and the trace identity tr(sum A A^T) = tr(sum A^T A)
    Xt = np.ascontiguousarray(np.swapaxes(X[:2000], 1, 2))
    _, _, _, c_rows = oracle.moments(X[:2000], X[:2000])
    _, _, _, c_cols = oracle.moments(Xt, Xt)
    np.testing.assert_allclose(np.trace(c_rows), np.trace(c_cols), rtol=1e-12)


# ------------------------------------------------------- P3: gain, update
def _random_spd(rng, p, cond=50.0):
    Q, _ = np.linalg.qr(rng.standard_normal((p, p)))
    ev = np.geomspace(1.0, cond, p)
    return (Q * ev) @ Q.T


def test_cholesky_matches_numpy():
    rng = np.random.default_rng(31)
    for p in (1, 2, 7, 20):
        A = _random_spd(rng, p)
        np.testing.assert_allclose(oracle.cholesky(A), np.linalg.cholesky(A), atol=1e-12)


def test_gain_matches_numpy_solve():
    rng = np.random.default_rng(32)
    for R, p in [(5, 3), (30, 20), (1, 1)]:
        A = _random_spd(rng, p, cond=1e3)
        C = rng.standard_normal((R, p))
        np.testing.assert_allclose(oracle.gain(C, A), np.linalg.solve(A, C.T).T, rtol=1e-10,
                                   atol=1e-12)


def test_gain_reports_not_positive_definite():
    A = np.diag([1.0, -1.0, 2.0])
    with pytest.raises(np.linalg.LinAlgError):
        oracle.gain(np.ones((2, 3)), A)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky(np.zeros((2, 2)))


def _textbook_enkf(Xv, Yv, ybar):
    """Perturbed-observation ensemble Kalman update for vectors (m = 1):
    rows of Xv/Yv are members; covariances from np.cov (1/(N-1)), gain from
    np.linalg.solve."""
    N, R = Xv.shape
    C = np.cov(Xv.T, Yv.T)                       # (R+p) x (R+p), ddof = 1
    Pxy, Pyy = C[:R, R:], C[R:, R:]
    K = np.linalg.solve(Pyy, Pxy.T).T
    return Xv + (ybar[None, :] - Yv) @ K.T, K


def test_analysis_m1_equals_textbook_vector_enkf():
    rng = np.random.default_rng(33)
    N, R, p = 40, 9, 4
    X = rng.standard_normal((N, R, 1))
    obs = [0, 2, 5, 8]
    V = 0.3 * rng.standard_normal((N, p, 1))
    Y = X[:, obs, :] + V
    ybar = rng.standard_normal((p, 1))
    got = oracle.enks_analysis(X, Y, ybar)
    want, _ = _textbook_enkf(X[:, :, 0], Y[:, :, 0], ybar[:, 0])
    np.testing.assert_allclose(got[:, :, 0], want, rtol=1e-10, atol=1e-12)


def test_analysis_mean_is_linear_in_innovation():
    # K does not depend on Ybar, so shifting Ybar by alpha*delta shifts the
    # posterior mean by alpha * K delta exactly.
    rng = np.random.default_rng(34)
    N, R, p, m = 30, 6, 3, 5
    X = rng.standard_normal((N, R, m))
    Y = X[:, :p, :] + 0.2 * rng.standard_normal((N, p, m))
    ybar = rng.standard_normal((p, m))
    delta = rng.standard_normal((p, m))
    a = oracle.enks_analysis(X, Y, ybar).mean(0)
    b = oracle.enks_analysis(X, Y, ybar + 2.5 * delta).mean(0)
    # K from numpy, pooled over columns (independent of the oracle)
    Ax = X - X.mean(0)
    Ay = Y - Y.mean(0)
    cxy = np.einsum("irj,icj->rc", Ax, Ay)
    cyy = np.einsum("irj,icj->rc", Ay, Ay)
    K = np.linalg.solve(cyy, cxy.T).T
    np.testing.assert_allclose(b - a, 2.5 * K @ delta, atol=1e-11)


# ------------------------------------------- P4/P5/P6: whole-solve pins
def _vertical_linear_net(n, m, l, rng):
    """One linear conv layer 2 -> 1 with only the centre column of taps (no
    horizontal coupling), so CNN_theta is x_{t+1} = A x_t + G u_t column-wise."""
    w = np.zeros((1, 2, 3, 3))
    w[0, 0, :, 1] = [0.15, -0.3, 0.1]
    w[0, 1, :, 1] = [0.2, 0.5, -0.1]
    B = rng.standard_normal((n, l))
    net = oracle.Net(n, m, l, [2, 1], [(w, np.zeros(1))], B, residual_scale=1.0)
    T = lambda taps: (np.diag(np.full(n, taps[1])) + np.diag(np.full(n - 1, taps[0]), -1)
                      + np.diag(np.full(n - 1, taps[2]), 1))
    A = np.eye(n) + T(w[0, 0, :, 1])
    G = T(w[0, 1, :, 1]) @ B
    return net, A, G


def _exact_smoother_ls(A, G, x_k, u_prev, xref, uref, H, sw, svx, svu):
    """Posterior mean of u_k, w_k..w_{k+H-1} for one column by weighted least
    squares (linear-Gaussian MAP = mean), then the smoothed controls
    u_k .. u_{k+H}.  Theorem 1: this is also the MPC optimum of J."""
    n, l = G.shape
    nz = (H + 1) * l
    rows, rhs = [], []
    # prior: u_k ~ N(u_prev, sw^2 I), w ~ N(0, sw^2 I)
    for i in range(nz):
        e = np.zeros(nz); e[i] = 1.0 / sw
        rows.append(e); rhs.append((u_prev[i] if i < l else 0.0) / sw)
    # u_{k+s} = Mu[s] z ; x_{k+s} = Ax[s] x_k + Mx[s] z
    Mu = [np.hstack([np.eye(l)] + [np.zeros((l, l))] * H)]
    Mx = [np.zeros((n, nz))]
    Ap = [np.eye(n)]
    for s in range(1, H + 1):
        Mx.append(A @ Mx[-1] + G @ Mu[-1])
        nxt = Mu[-1].copy()
        nxt[:, s * l:(s + 1) * l] += np.eye(l)
        Mu.append(nxt)
        Ap.append(A @ Ap[-1])
    for s in range(1, H + 1):
        for r in range(n):
            rows.append(Mx[s][r] / svx); rhs.append((xref[s][r] - (Ap[s] @ x_k)[r]) / svx)
        for r in range(l):
            rows.append(Mu[s][r] / svu); rhs.append(uref[r] / svu)
    z, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    return np.stack([Mu[s] @ z for s in range(H + 1)])


@pytest.mark.parametrize("N", [4000])
def test_solve_linear_gaussian_converges_to_exact_smoother(N):
    rng = np.random.default_rng(41)
    n, m, l, H = 6, 16, 2, 3
    sw, svx, svu = 0.3, 0.2, 0.5
    net, A, G = _vertical_linear_net(n, m, l, rng)
    x_k = rng.standard_normal((n, m))
    u_prev = 0.5 * rng.standard_normal((l, m))
    xref = rng.standard_normal((H + 1, n, m))
    uref = np.zeros((l, m))
    nr = np.random.default_rng(42)
    noise = np.concatenate([
        (sw * nr.standard_normal((N, l, m))).ravel(), (sw * nr.standard_normal((H, N, l, m))).ravel(),
        (svx * nr.standard_normal((H, N, n, m))).ravel(), (svu * nr.standard_normal((H, N, l, m))).ravel()])
    xh = oracle.enks_solve(net, N, H, x_k, u_prev, xref, uref, noise)
    U_enks = xh[:, n:n + l, :]
    U_exact = np.stack([_exact_smoother_ls(A, G, x_k[:, j], u_prev[:, j], xref[:, :, j],
                                           uref[:, j], H, sw, svx, svu) for j in range(m)], axis=-1)
    # sampling error of an N*m-sample ensemble: a few percent of the prior spread
    err = np.abs(U_enks - U_exact).max()
    assert err < 0.05 * sw * 3, err
    # and the smoother moved the controls well beyond that error
    assert np.abs(U_exact - u_prev[None]).max() > 10 * err
    # ensemble X_k block is never updated (zero anomaly)
    np.testing.assert_allclose(xh[0, :n], x_k, atol=1e-12)
    # dU_k = U_k - U_{k-1} holds for the smoothed means (identical anomalies)
    np.testing.assert_allclose(xh[0, n + l:], xh[0, n:n + l] - u_prev, atol=1e-10)


def _vector_enks_solve(net, N, H, x_k, u_prev, xref, uref, noise):
    """Textbook single-pass EnKS on the vectorised augmented state for m = 1,
    written independently: each member is a flat vector holding blocks k..t of
    [x; u; du]; the update uses np.cov and np.linalg.solve."""
    n, l = net.n, net.l
    q, p = n + 2 * l, n + l
    W0 = noise[:N * l].reshape(N, l)
    off = N * l
    Wn = noise[off:off + H * N * l].reshape(H, N, l); off += H * N * l
    VX = noise[off:off + H * N * n].reshape(H, N, n); off += H * N * n
    VU = noise[off:off + H * N * l].reshape(H, N, l)
    ens = np.concatenate([np.tile(x_k, (N, 1)), u_prev[None] + W0, W0], axis=1)  # N x q
    for s in range(1, H + 1):
        last = ens[:, -q:]
        xn = np.stack([oracle.cnn_step(net, last[i, :n, None], last[i, n:n + l, None])[:, 0]
                       for i in range(N)])
        blk = np.concatenate([xn, last[:, n:n + l] + Wn[s - 1], Wn[s - 1]], axis=1)
        ens = np.concatenate([ens, blk], axis=1)
        Y = np.concatenate([blk[:, :n] + VX[s - 1], blk[:, n:n + l] + VU[s - 1]], axis=1)
        ybar = np.concatenate([xref[s], uref])
        ens, _ = _textbook_enkf(ens, Y, ybar)
    return ens.mean(0).reshape(H + 1, q)


def test_solve_m1_equals_textbook_vector_enks():
    rng = np.random.default_rng(51)
    n, l, N, H = 8, 3, 24, 4
    ws = [(0.3 * rng.standard_normal((8, 2, 3, 3)), 0.1 * rng.standard_normal(8)),
          (0.3 * rng.standard_normal((1, 8, 3, 3)), np.zeros(1))]
    net = oracle.Net(n, 1, l, [2, 8, 1], ws, rng.standard_normal((n, l)))
    x_k = rng.standard_normal(n)
    u_prev = rng.standard_normal(l)
    xref = rng.standard_normal((H + 1, n))
    uref = rng.standard_normal(l)
    noise = 0.1 * rng.standard_normal(oracle.noise_floats(n, 1, l, N, H))
    got = oracle.enks_solve(net, N, H, x_k[:, None], u_prev[:, None], xref[:, :, None],
                            uref[:, None], noise)[:, :, 0]
    want = _vector_enks_solve(net, N, H, x_k, u_prev, xref, uref, noise)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-10)


# --------------------------------------------------------- cost and P7
def test_cost_trace_form_equals_vec_kronecker_form():
    # Problem Setup: tr[(X-Xr)^T R^{-1} (X-Xr)] = vec(X-Xr)^T (I kron R)^{-1} vec(X-Xr)
    rng = np.random.default_rng(61)
    n, m = 4, 3
    D = rng.standard_normal((n, m))
    Rm = _random_spd(rng, n, 5.0)
    tr_form = np.trace(D.T @ np.linalg.inv(Rm) @ D)
    vec = D.ravel(order="F")
    kron_form = vec @ np.linalg.inv(np.kron(np.eye(m), Rm)) @ vec
    assert abs(tr_form - kron_form) < 1e-10 * abs(tr_form)
    # the isotropic case used by the oracle's closed_loop_cost
    s = 0.01
    Xr = np.zeros((2, n, m)); Xt = np.stack([np.zeros((n, m)), D])
    c = oracle.closed_loop_cost(Xt, np.zeros((1, 1, m)), Xr, np.zeros((1, m)), np.zeros((1, m)), s, s, s)
    assert abs(c - np.sum(D ** 2) / s ** 2) < 1e-8 * c


def test_golden_closed_loop_cost_hand_worked():
    """J with non-zero state, control and increment terms over S = 2 steps:
    an off-by-one in the reference window, the control reference or the
    U_{-1} = U_init increment changes the value."""
    for c in json.load(open(os.path.join(GOLDEN, "closed_loop_cost.json")))["cases"]:
        J = oracle.closed_loop_cost(np.array(c["X_traj"]), np.array(c["U_traj"]), np.array(c["X_ref_all"]),
                                    np.array(c["U_ref"]), np.array(c["U_init"]), c["sigma_vx"], c["sigma_vu"],
                                    c["sigma_w"])
        assert abs(J - c["J"]) <= 1e-12 * c["J"], (J, c["J"])


def test_run_applies_the_theorem1_optimum_of_each_window():
    """Algorithm 1's receding loop against Theorem 1.  With a vertical-tap
    linear CNN (x_{t+1} = A x_t + G u_t per column) and isotropic Gaussian
    noise, the smoother's mean at each control step k is the weighted
    least-squares optimum of J over the window k..k+H, solved from the plant
    state X_k and the last applied control U_{k-1}.  So, for a non-zero,
    time-varying reference and a non-zero U^ref:
      * every applied control U_k is within sampling error of the optimum's
        first control u_k (not of u_{k+1}, and not of the optimum for the
        window k+1..k+H+1 or for a stale U_{k-1});
      * every returned plan U_hat[k] is within sampling error of the optimum;
      * the plant advances by the exact linear map X_{k+1} = A X_k + G U_k.
    The alternatives are checked to lie far outside the tolerance, so a wrong
    window offset, block or warm start fails this test."""
    rng = np.random.default_rng(71)
    n, m, l, H, S, N = 6, 16, 2, 3, 3, 16000
    sw, svx, svu = 0.3, 0.2, 0.5
    net, A, G = _vertical_linear_net(n, m, l, rng)
    x0 = rng.standard_normal((n, m))
    u_init = 0.5 * rng.standard_normal((l, m))
    xref_all = rng.standard_normal((S + H + 1, n, m))
    uref = 0.3 * rng.standard_normal((l, m))
    nr = np.random.default_rng(72)
    noise_all = np.stack([np.concatenate([
        (sw * nr.standard_normal((N, l, m))).ravel(), (sw * nr.standard_normal((H, N, l, m))).ravel(),
        (svx * nr.standard_normal((H, N, n, m))).ravel(), (svu * nr.standard_normal((H, N, l, m))).ravel()])
        for _ in range(S)])
    Xt, Ut, Uh = oracle.run(net, N, H, S, x0, u_init, xref_all, uref, noise_all)

    def optimum(xk, up, xr):
        return np.stack([_exact_smoother_ls(A, G, xk[:, j], up[:, j], xr[:, :, j], uref[:, j], H, sw, svx, svu)
                         for j in range(m)], axis=-1)

    tol = 0.05 * sw * 3
    np.testing.assert_array_equal(Xt[0], x0)
    up = u_init
    for k in range(S):
        np.testing.assert_allclose(Xt[k + 1], A @ Xt[k] + G @ Ut[k], rtol=0, atol=1e-12)
        opt = optimum(Xt[k], up, xref_all[k:k + H + 1])
        assert np.abs(Ut[k] - opt[0]).max() < tol
        assert np.abs(Uh[k] - opt).max() < tol
        np.testing.assert_array_equal(Uh[k][0], Ut[k])
        later_window = optimum(Xt[k], up, xref_all[k + 1:k + H + 2])[0]
        assert np.abs(opt[1] - opt[0]).max() > 4 * tol
        assert np.abs(later_window - opt[0]).max() > 4 * tol
        if k > 0:
            assert np.abs(optimum(Xt[k], u_init, xref_all[k:k + H + 1])[0] - opt[0]).max() > 4 * tol
        up = Ut[k]


@pytest.mark.slow
def test_closed_loop_cost_below_uncontrolled():
    # Numerical Experiments: under Kalman-MPC the tracking error falls and the
    # cost J is lower than with no control.  The 16 x 16 fixture's B ~ N(0, 0.1^2)
    # gives the control almost no authority over X (its effect is far below the
    # 0.01 pseudo-noise), so this pin uses the same CNN with B ~ N(0, 1), a
    # wider exploration sigma_w = 0.05 and a cheaper control sigma_vu = 0.1,
    # where control pays.
    wl = W.small_16().with_(sigma_w=0.05, sigma_vu=0.1)
    net = oracle.Net(wl.n, wl.m, wl.l, wl.channels, wl.weights(), 10.0 * wl.B())
    S = wl.S
    xr = wl.X_ref_all(S)
    Xt, Ut, _ = oracle.run(net, wl.N, wl.H, S, wl.X0(), wl.U_init(), xr, wl.U_ref(),
                           wl.noise_all(S))
    j_ctl = oracle.closed_loop_cost(Xt, Ut, xr, wl.U_ref(), wl.U_init(), wl.sigma_vx, wl.sigma_vu,
                                    wl.sigma_w)
    X0 = np.zeros_like(Xt)
    X0[0] = wl.X0()
    for k in range(S):
        X0[k + 1] = oracle.cnn_step(net, X0[k], np.zeros((wl.l, wl.m)))
    j_free = oracle.closed_loop_cost(X0, np.zeros_like(Ut), xr, wl.U_ref(), wl.U_init(),
                                     wl.sigma_vx, wl.sigma_vu, wl.sigma_w)
    assert j_ctl < 0.95 * j_free, (j_ctl, j_free)
    # tracking error (zero reference) ends lower than without control
    assert oracle.rmse(Xt[-1], xr[S]) < oracle.rmse(X0[-1], xr[S])


# ---------------------------------------------------------------- narrow controls
# The right transformation of the paragraph after Table I: U = u T, and back
# u = U T^T (T T^T)^{-1}.

def test_control_expand_hand_worked():
    u = np.array([[1.0, 2.0], [-1.0, 0.5]])
    T = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 1.0]])
    np.testing.assert_array_equal(oracle.control_expand(u, T), [[1.0, 2.0, 3.0], [-1.0, 0.5, -0.5]])


def test_control_reduce_with_ones_row_is_the_column_mean():
    """T = [1 ... 1] repeats a column vector; the map back is the mean over
    the columns: U 1^T / m."""
    rng = np.random.default_rng(1)
    U = rng.standard_normal((5, 12))
    u = oracle.control_reduce(U, np.ones((1, 12)))
    np.testing.assert_allclose(u[:, 0], U.mean(axis=1), rtol=0, atol=1e-14)


def test_control_reduce_inverts_expand_and_identity():
    rng = np.random.default_rng(2)
    for mu, m in ((1, 8), (3, 16), (7, 64)):
        T = rng.standard_normal((mu, m))
        u = rng.standard_normal((4, mu))
        np.testing.assert_allclose(oracle.control_reduce(oracle.control_expand(u, T), T), u, rtol=0, atol=1e-12)
    U = rng.standard_normal((3, 9))
    np.testing.assert_allclose(oracle.control_reduce(U, np.eye(9)), U, rtol=0, atol=1e-14)
    np.testing.assert_allclose(oracle.control_expand(U, np.eye(9)), U, rtol=0, atol=0)


def test_control_reduce_reports_rank_deficient_transform():
    T = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0]])      # T T^T singular
    with pytest.raises(np.linalg.LinAlgError):
        oracle.control_reduce(np.ones((2, 3)), T)

"""FP64 CPU oracle for Kalman-MPC (arXiv 2410.09663) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never touches it and it
never touches the CUDA library: the two share no code.  The arithmetic lives in
``oracle.c`` (plain C, double precision, written from the paper's equations);
this module compiles it with gcc, loads it with ctypes and converts arrays.

Parity status per function (see the tests that pin each one):
  cnn_step        pinned: numpy im2col + matmul, scipy correlate2d, analytic
                  discrete Laplacian of a quadratic field
  moments         pinned: two-member hand formula, permutation invariance,
                  trace identity of the Appendix moments
  gain            pinned: numpy Cholesky / solve on random SPD matrices
  enks_analysis   pinned: textbook vector EnKF (m = 1), linearity of the mean
                  in the innovation, lambda / normalisation invariance
  enks_solve      pinned: exact linear-Gaussian smoother = weighted least squares
                  (Theorem 1) for a vertical-tap linear CNN, as N*m grows
  run             pinned: for a vertical-tap linear CNN and a non-zero,
                  time-varying reference, every applied control is the first
                  control of the Theorem-1 least-squares optimum over the
                  window k..k+H from the current plant state and the last
                  applied control, and the plant moves by the exact linear
                  map; closed-loop cost under control below the uncontrolled
                  cost (qualitative, Numerical Experiments section)
  closed_loop_cost pinned: a hand-worked S = 2 case with non-zero state,
                  control and increment terms (tests/golden/closed_loop_cost.json)
  control_expand  pinned: a hand-worked product, T = I
  control_reduce  pinned: column means for T = [1 ... 1], reduce(expand(u)) = u,
                  T = I, rank-deficient T reported
  softplus_barrier pinned: closed forms phi(0) = ln 2 / alpha,
                  phi(ln(e - 1) / beta) = 1 / alpha, phi(x) - phi(-x) = beta x / alpha,
                  the two limits (0 far inside, beta x / alpha far outside)
  constraint_obs  pinned: a hand-worked 2-row case
  row_cov         pinned: numpy's biased per-column covariance summed over the
                  columns, the lambda factor
  enks_solve_cov  pinned: an H = 1 solve rebuilt from pinned pieces (CNN step,
                  row_cov, textbook analysis), and the exact sample identity
                  Sigma_post = Sigma_pred - S_XY S_Y^{-1} S_YX of the perturbed-
                  observation update (the "-" sign of the Appendix)
  enks_solve / run with constraints: pinned by an H = 1 solve rebuilt from the
                  pinned pieces (CNN step, constraint rows, textbook analysis)
                  and by a solve whose control reference lies outside a box:
                  the plan follows it without the rows and sits at the bound
                  with them (sign and strength of the barrier's pull)
  nonlinear multi-layer solves beyond these pins: parity unpinned -- the oracle
  itself is the authority there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
MAX_LAYERS = 8


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP over members)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


class _Net(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("m", ctypes.c_int), ("l", ctypes.c_int),
        ("n_layers", ctypes.c_int),
        ("channels", ctypes.c_int * (MAX_LAYERS + 1)),
        ("w", ctypes.POINTER(ctypes.c_double)),
        ("b", ctypes.POINTER(ctypes.c_double)),
        ("B", ctypes.POINTER(ctypes.c_double)),
        ("residual_scale", ctypes.c_double),
    ]


class _Cons(ctypes.Structure):
    _fields_ = [
        ("c", ctypes.c_int),
        ("Gx", ctypes.POINTER(ctypes.c_double)),
        ("Gu", ctypes.POINTER(ctypes.c_double)),
        ("h", ctypes.POINTER(ctypes.c_double)),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER(ctypes.c_double)
        i, l_ = ctypes.c_int, ctypes.c_long
        _lib.oracle_conv3x3.argtypes = [i, i, i, i, P, P, P, i, P]
        _lib.oracle_cnn_step.argtypes = [ctypes.POINTER(_Net), P, P, P]
        _lib.oracle_cnn_step_batch.argtypes = [ctypes.POINTER(_Net), i, P, P, P]
        _lib.oracle_moments.argtypes = [i, i, i, i, P, l_, P, P, P, P, P]
        _lib.oracle_cholesky.argtypes = [i, P, P]
        _lib.oracle_gain.argtypes = [i, i, P, P, P]
        _lib.oracle_enks_analysis.argtypes = [i, i, i, i, P, l_, P, P]
        _lib.oracle_enks_solve.argtypes = [ctypes.POINTER(_Net), i, i, P, P, P, P, P, P]
        _lib.oracle_run.argtypes = [ctypes.POINTER(_Net), i, i, i, P, P, P, P, P, P, P, P]
        _lib.oracle_control_expand.argtypes = [i, i, i, P, P, P]
        _lib.oracle_control_expand.restype = None
        _lib.oracle_control_reduce.argtypes = [i, i, i, P, P, P]
        C = ctypes.POINTER(_Cons)
        _lib.oracle_softplus_barrier.argtypes = [ctypes.c_double] * 3
        _lib.oracle_softplus_barrier.restype = ctypes.c_double
        _lib.oracle_constraint_obs.argtypes = [C, i, i, i, P, P, P, P]
        _lib.oracle_constraint_obs.restype = None
        _lib.oracle_enks_solve_c.argtypes = [ctypes.POINTER(_Net), i, i, P, P, P, P, P, C, P]
        _lib.oracle_run_c.argtypes = [ctypes.POINTER(_Net), i, i, i, P, P, P, P, P, C, P, P, P]
        _lib.oracle_row_cov.argtypes = [i, i, i, P, l_, ctypes.c_double, P]
        _lib.oracle_enks_solve_cov.argtypes = [ctypes.POINTER(_Net), i, i, P, P, P, P, P, C, ctypes.c_double,
                                               P, P, P]
        for f in ("oracle_cnn_step", "oracle_cnn_step_batch", "oracle_cholesky", "oracle_gain",
                  "oracle_enks_analysis", "oracle_enks_solve", "oracle_run", "oracle_control_reduce",
                  "oracle_enks_solve_c", "oracle_run_c", "oracle_row_cov", "oracle_enks_solve_cov"):
            getattr(_lib, f).restype = ctypes.c_int
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Net:
    """CNN_theta of Eq. (1) in the oracle's FP64 representation.

    ``weights`` is a list of (w [Cout][Cin][3][3], b [Cout]) per layer; ``B`` is
    n x l.  Values are converted to float64 exactly (the tests pass the same
    float32 numbers the GPU receives).
    """

    def __init__(self, n, m, l, channels, weights, B, residual_scale=0.1):
        assert len(channels) == len(weights) + 1 and len(weights) <= MAX_LAYERS
        self.n, self.m, self.l = int(n), int(m), int(l)
        self.channels = [int(c) for c in channels]
        self._w = _d(np.concatenate([np.asarray(w, np.float64).ravel() for w, _ in weights]))
        self._b = _d(np.concatenate([np.asarray(b, np.float64).ravel() for _, b in weights]))
        self._B = _d(np.asarray(B, np.float64).reshape(n, l))
        self.residual_scale = float(residual_scale)
        s = _Net()
        s.n, s.m, s.l, s.n_layers = self.n, self.m, self.l, len(weights)
        for k, c in enumerate(self.channels):
            s.channels[k] = c
        s.w, s.b, s.B = _p(self._w), _p(self._b), _p(self._B)
        s.residual_scale = self.residual_scale
        self._s = s

    @property
    def q(self):
        return self.n + 2 * self.l

    @property
    def p(self):
        return self.n + self.l


class Cons:
    """c virtual constraint observations z = phi(Gx X + Gu U - h 1^T) + eps with
    reference 0, phi(x) = ln(1 + e^{beta x}) / alpha (the paragraph on
    state/input constraints after Table I).  Gx: c x n, Gu: c x l, h: c."""

    def __init__(self, Gx, Gu, h, alpha, beta):
        self.Gx = _d(np.atleast_2d(Gx))
        self.Gu = _d(np.atleast_2d(Gu))
        self.h = _d(np.ravel(h))
        self.c = self.h.size
        assert self.Gx.shape[0] == self.c and self.Gu.shape[0] == self.c
        self.alpha, self.beta = float(alpha), float(beta)
        s = _Cons()
        s.c = self.c
        s.Gx, s.Gu, s.h = _p(self.Gx), _p(self.Gu), _p(self.h)
        s.alpha, s.beta = self.alpha, self.beta
        self._s = s


def _cons_ptr(cons):
    return ctypes.byref(cons._s) if cons is not None else None


def softplus_barrier(x, alpha, beta):
    """phi(x) = ln(1 + e^{beta x}) / alpha, element-wise."""
    f = _load().oracle_softplus_barrier
    x = np.asarray(x, np.float64)
    return np.vectorize(lambda v: f(float(v), float(alpha), float(beta)))(x) if x.ndim else f(float(x), alpha, beta)


def constraint_obs(cons: Cons, X, U, eps=None):
    """z = phi(Gx X + Gu U - h 1^T) + eps for one member (X: n x m, U: l x m)."""
    X, U = _d(X), _d(U)
    n, m = X.shape
    l = U.shape[0]
    assert cons.Gx.shape[1] == n and cons.Gu.shape[1] == l
    eps = np.zeros((cons.c, m)) if eps is None else _d(eps).reshape(cons.c, m)
    z = np.empty((cons.c, m))
    _load().oracle_constraint_obs(ctypes.byref(cons._s), n, l, m, _p(X), _p(U), _p(eps), _p(z))
    return z


def conv3x3(x, w, b, apply_tanh=False):
    """One 3x3 'same' conv layer: x [Cin][n][m], w [Cout][Cin][3][3], b [Cout]."""
    x, w, b = _d(x), _d(w), _d(b)
    cin, n, m = x.shape
    cout = w.shape[0]
    out = np.empty((cout, n, m))
    _load().oracle_conv3x3(cin, cout, n, m, _p(x), _p(w), _p(b), int(bool(apply_tanh)), _p(out))
    return out


def cnn_step(net: Net, X, U):
    """X_{k+1} = CNN_theta(X_k, U_k), Eq. (1); X [..., n, m], U [..., l, m]."""
    X, U = _d(X), _d(U)
    batch_shape = X.shape[:-2]
    Xb = X.reshape(-1, net.n, net.m)
    Ub = _d(U.reshape(-1, net.l, net.m))
    out = np.empty_like(Xb)
    st = _load().oracle_cnn_step_batch(ctypes.byref(net._s), Xb.shape[0], _p(Xb), _p(Ub), _p(out))
    if st:
        raise MemoryError("oracle_cnn_step failed")
    return out.reshape(batch_shape + (net.n, net.m))


def moments(X, Y):
    """Means and covariances of Eq. (Ybar-sample-mean-cov), lambda = 1.

    X [N][R][m], Y [N][p][m] -> (xmean, ymean, Cxy, Cyy)."""
    X, Y = _d(X), _d(Y)
    N, R, m = X.shape
    p = Y.shape[1]
    xm, ym = np.empty((R, m)), np.empty((p, m))
    cxy, cyy = np.empty((R, p)), np.empty((p, p))
    _load().oracle_moments(N, R, p, m, _p(X), R * m, _p(Y), _p(xm), _p(ym), _p(cxy), _p(cyy))
    return xm, ym, cxy, cyy


def cholesky(A):
    A = _d(A)
    L = np.empty_like(A)
    st = _load().oracle_cholesky(A.shape[0], _p(A), _p(L))
    if st:
        raise np.linalg.LinAlgError(f"not positive definite at pivot {st - 1}")
    return L


def gain(Cxy, Cyy):
    """K = Cxy Cyy^{-1}."""
    Cxy, Cyy = _d(Cxy), _d(Cyy)
    K = np.empty_like(Cxy)
    st = _load().oracle_gain(Cxy.shape[0], Cyy.shape[0], _p(Cxy), _p(Cyy), _p(K))
    if st:
        raise np.linalg.LinAlgError(f"Cyy not positive definite (status {st})")
    return K


def enks_analysis(X, Y, Ybar):
    """Member-wise update X^i + K (Ybar - Y^i); returns the updated copy."""
    X = _d(X).copy()
    Y, Ybar = _d(Y), _d(Ybar)
    N, R, m = X.shape
    p = Y.shape[1]
    st = _load().oracle_enks_analysis(N, R, p, m, _p(X), R * m, _p(Y), _p(Ybar))
    if st:
        raise np.linalg.LinAlgError(f"analysis failed (status {st})")
    return X


def noise_floats(n, m, l, N, H, c=0):
    """Length of one solve's noise buffer: W0, W, VX, VU (and VZ for c
    constraint rows)."""
    return N * l * m + H * N * (l * m + n * m + l * m + c * m)


def enks_solve(net: Net, N, H, X_k, U_prev, X_ref, U_ref, noise, cons: Cons | None = None):
    """One receding-horizon solve (Algorithm 1, one control step) with full history,
    with the constraint rows of `cons` appended to the pseudo-observation.

    Returns Xbar_hat [(H+1)][q][m]: smoothed means of blocks k..k+H."""
    n, m, l = net.n, net.m, net.l
    X_k, U_prev, U_ref = _d(X_k), _d(U_prev), _d(U_ref)
    X_ref = _d(X_ref).reshape(H + 1, n, m)
    noise = _d(noise).ravel()
    assert noise.size == noise_floats(n, m, l, N, H, cons.c if cons is not None else 0)
    out = np.empty((H + 1, net.q, m))
    st = _load().oracle_enks_solve_c(ctypes.byref(net._s), N, H, _p(X_k), _p(U_prev), _p(X_ref),
                                     _p(U_ref), _p(noise), _cons_ptr(cons), _p(out))
    if st:
        raise np.linalg.LinAlgError(f"solve failed (status {st})")
    return out


def row_cov(X, lam=1.0):
    """(lam / N) sum_i (X^i - Xhat)(X^i - Xhat)^T for X [N][R][m] (R x R)."""
    X = _d(X)
    N, R, m = X.shape
    S = np.empty((R, R))
    if _load().oracle_row_cov(N, R, m, _p(X), R * m, float(lam), _p(S)):
        raise MemoryError("oracle_row_cov")
    return S


def enks_solve_cov(net: Net, N, H, X_k, U_prev, X_ref, U_ref, noise, cons: Cons | None = None, lam=1.0):
    """enks_solve with Algorithm 1's optional covariance steps executed.

    Returns (Xbar_hat, pred, post): pred[s-1] / post[s-1] is the (s+1) q x
    (s+1) q row covariance (factor lam / N) of the history blocks 0..s after
    the prediction to t = k+s and after the update at t."""
    n, m, l = net.n, net.m, net.l
    X_k, U_prev, U_ref = _d(X_k), _d(U_prev), _d(U_ref)
    X_ref = _d(X_ref).reshape(H + 1, n, m)
    noise = _d(noise).ravel()
    assert noise.size == noise_floats(n, m, l, N, H, cons.c if cons is not None else 0)
    Rf = (H + 1) * net.q
    out = np.empty((H + 1, net.q, m))
    pred = np.zeros((H, Rf * Rf))
    post = np.zeros((H, Rf * Rf))
    st = _load().oracle_enks_solve_cov(ctypes.byref(net._s), N, H, _p(X_k), _p(U_prev), _p(X_ref), _p(U_ref),
                                       _p(noise), _cons_ptr(cons), float(lam), _p(pred), _p(post), _p(out))
    if st:
        raise np.linalg.LinAlgError(f"solve failed (status {st})")
    sl = lambda a, s: a[s - 1, :((s + 1) * net.q) ** 2].reshape((s + 1) * net.q, (s + 1) * net.q)
    return out, [sl(pred, s) for s in range(1, H + 1)], [sl(post, s) for s in range(1, H + 1)]


def run(net: Net, N, H, S, X_0, U_init, X_ref_all, U_ref, noise_all, cons: Cons | None = None):
    """S receding-horizon steps (Algorithm 1), plant = CNN_theta.

    X_ref_all holds references for absolute times 0 .. S+H-1 (at least S+H
    blocks).  Returns (X_traj [S+1][n][m], U_traj [S][l][m],
    U_hat_all [S][H+1][l][m])."""
    n, m, l = net.n, net.m, net.l
    X_0, U_init, U_ref = _d(X_0), _d(U_init), _d(U_ref)
    X_ref_all = _d(X_ref_all).reshape(-1, n, m)
    assert X_ref_all.shape[0] >= S + H
    noise_all = _d(noise_all).ravel()
    assert noise_all.size == S * noise_floats(n, m, l, N, H, cons.c if cons is not None else 0)
    Xt = np.empty((S + 1, n, m))
    Ut = np.empty((S, l, m))
    Uh = np.empty((S, H + 1, l, m))
    st = _load().oracle_run_c(ctypes.byref(net._s), N, H, S, _p(X_0), _p(U_init), _p(X_ref_all),
                              _p(U_ref), _p(noise_all), _cons_ptr(cons), _p(Xt), _p(Ut), _p(Uh))
    if st:
        raise np.linalg.LinAlgError(f"run failed (status {st})")
    return Xt, Ut, Uh


def closed_loop_cost(X_traj, U_traj, X_ref_all, U_ref, U_init, sigma_vx, sigma_vu, sigma_w):
    """Tracking cost J of the Problem Setup section evaluated on the applied
    trajectory with isotropic weights R = sigma_vx^2 I, Q_U = sigma_vu^2 I,
    Q_dU = sigma_w^2 I:

      J = sum_{k=1}^{S} ||X_k - X^ref_k||_F^2 / sigma_vx^2
        + sum_{k=0}^{S-1} ( ||U_k - U^ref||_F^2 / sigma_vu^2
                          + ||U_k - U_{k-1}||_F^2 / sigma_w^2 ),   U_{-1} = U_init.
    """
    X_traj, U_traj = _d(X_traj), _d(U_traj)
    S = U_traj.shape[0]
    Xr = _d(X_ref_all)[1:S + 1]
    jx = np.sum((X_traj[1:S + 1] - Xr) ** 2) / sigma_vx ** 2
    ju = np.sum((U_traj - _d(U_ref)[None]) ** 2) / sigma_vu ** 2
    prev = np.concatenate([_d(U_init)[None], U_traj[:-1]], axis=0)
    jd = np.sum((U_traj - prev) ** 2) / sigma_w ** 2
    return float(jx + ju + jd)


def rmse(X, X_ref):
    """Tracking RMSE diagnostic sqrt(||X - X_ref||_F^2 / (n m))."""
    X, X_ref = _d(X), _d(X_ref)
    return float(np.sqrt(np.mean((X - X_ref) ** 2)))


def control_expand(u, T):
    """Narrow controls: U = u T (u: l x mu, T: mu x m)."""
    u, T = _d(u), _d(T)
    U = np.empty((u.shape[0], T.shape[1]))
    _load().oracle_control_expand(u.shape[0], u.shape[1], T.shape[1], _p(u), _p(T), _p(U))
    return U


def control_reduce(U, T):
    """Narrow controls: u = U T^T (T T^T)^{-1} (U: l x m, T: mu x m)."""
    U, T = _d(U), _d(T)
    u = np.empty((U.shape[0], T.shape[0]))
    st = _load().oracle_control_reduce(U.shape[0], U.shape[1], T.shape[0], _p(U), _p(T), _p(u))
    if st:
        raise np.linalg.LinAlgError(f"T T^T not positive definite (status {st})")
    return u

"""GPU parity of Algorithm 1's optional covariance outputs (oic_solve_cov:
Sigma^X_{t|t-1} after every prediction and Sigma^X_{t|t} after every update,
over the rows the handle keeps) against the FP64 oracle.

Tolerance: relative L2 error <= 1e-3 per slot.  The covariances are
second moments of anomalies about 1% of the values they are taken from, so
the FP32 ensemble's rounding (held to 1e-4 on the means) is magnified by the
ratio of value to anomaly before the FP64 sums; the observed errors sit well
inside this bound.  The controls of the same call are held to the solve's own
1e-4 and must equal a plain oic_solve bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2410_09663_b300 as oic
from paper_2410_09663_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-4
TOL_COV = 1e-3

RAGGED = W.Workload("ragged_20x24", n=20, m=24, l=3, channels=[2, 6, 1], N=19, H=3, S=4, ref="blobs",
                    blob_sigma=3.0)
TC_RAGGED = W.Workload("tc_24x32", n=24, m=32, l=4, channels=[2, 32, 32, 1], N=13, H=3, S=3,
                       ref="blobs", blob_sigma=4.0)
CASES = {"small_16": W.small_16(), "ragged": RAGGED, "tc_ragged": TC_RAGGED,
         "small_16_box": W.small_16().with_(cons=W.u_box(16, 4, 0.1))}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def kept_rows(wl, s, full):
    """The oracle's history rows (blocks of q = n + 2l) that the handle keeps
    at s, in the handle's order."""
    q = wl.n + 2 * wl.l
    rows = []
    if full:
        for t in range(1, s + 1):
            rows += [t * q + y for y in range(wl.n)]
    else:
        rows += [s * q + y for y in range(wl.n)]
    for t in range(s + 1):
        rows += [t * q + wl.n + y for y in range(wl.l)]
    return np.array(rows)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("full", [False, True])
def test_covariance_outputs_match_oracle(cuda_ok, name, full):
    import torch
    wl = CASES[name]
    w, b = wl.flat_weights()
    s = oic.Solver(oic.config_from_workload(wl, keep_full_history=full), w, b, wl.B(), constraints=wl.cons)
    k, lam = 1, 0.5
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    Xk, Up = dev(wl.X0()), dev(0.01 * np.random.default_rng(5).standard_normal((wl.l, wl.m)))
    xr, ur, nz = dev(wl.X_ref_window(k)), dev(wl.U_ref()), dev(wl.noise(k))
    H = wl.H
    R = s.oic_cov_rows(H)
    pred = torch.zeros(H * R * R, dtype=torch.float64, device="cuda")
    post = torch.zeros_like(pred)
    U_hat = torch.zeros(H + 1, wl.l, wl.m, device="cuda")
    s.oic_solve_cov(Xk, Up, xr, ur, nz, U_hat, None, lam, pred, post)
    U_plain = torch.zeros_like(U_hat)
    s.oic_solve(Xk, Up, xr, ur, nz, U_plain)
    s.oic_sync()
    assert torch.equal(U_hat, U_plain)

    cons = (oracle.Cons(wl.cons.Gx, wl.cons.Gu, wl.cons.h, wl.cons.alpha, wl.cons.beta)
            if wl.cons is not None else None)
    net = oracle.Net(wl.n, wl.m, wl.l, wl.channels, wl.weights(), wl.B(), wl.residual_scale)
    xh, opred, opost = oracle.enks_solve_cov(net, wl.N, H, wl.X0(), Up.cpu().numpy(), wl.X_ref_window(k),
                                             wl.U_ref(), wl.noise(k), cons, lam=lam)
    assert rel(U_hat.cpu().numpy(), xh[:, wl.n:wl.n + wl.l]) <= TOL
    gp = pred.cpu().numpy().reshape(H, R * R)
    gq = post.cpu().numpy().reshape(H, R * R)
    for t in range(1, H + 1):
        r = s.oic_cov_rows(t)
        idx = kept_rows(wl, t, full)
        assert r == idx.size
        want_p = opred[t - 1][np.ix_(idx, idx)]
        want_q = opost[t - 1][np.ix_(idx, idx)]
        got_p = gp[t - 1, :r * r].reshape(r, r)
        got_q = gq[t - 1, :r * r].reshape(r, r)
        assert rel(got_p, want_p) <= TOL_COV, (t, rel(got_p, want_p))
        assert rel(got_q, want_q) <= TOL_COV, (t, rel(got_q, want_q))
        assert np.trace(got_q) < np.trace(got_p)            # the update shrinks the spread
    s.close()

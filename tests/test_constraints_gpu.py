"""GPU parity of the constraint rows (virtual observations z = phi(g(X_t,
U_t)) + eps with reference 0, the paragraph on state/input constraints after
Table I of arXiv 2410.09663) against the FP64 oracle, through the C ABI.

Tolerance: relative L2 error <= 1e-4 on the smoothed controls and fields, the
bar of the unconstrained FP32 path.  The cases push the plan against the
constraints (a control reference outside a box, random affine rows on X and
U), so the barrier's rows carry weight in every compared result."""
import numpy as np
import pytest

import oracle
import paper_2410_09663_b300 as oic
from paper_2410_09663_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-4

RAGGED = W.Workload("ragged_20x24", n=20, m=24, l=3, channels=[2, 6, 1], N=19, H=3, S=4, ref="blobs",
                    blob_sigma=3.0)
MID = W.Workload("mid_32x48", n=32, m=48, l=4, channels=[2, 16, 16, 1], N=64, H=4, S=3, ref="blobs",
                 blob_sigma=4.0)
TC_RAGGED = W.Workload("tc_24x32", n=24, m=32, l=4, channels=[2, 32, 32, 1], N=13, H=3, S=3,
                       ref="blobs", blob_sigma=4.0)
CASES = {"small_16": W.small_16(), "ragged": RAGGED, "mid": MID, "tc_ragged": TC_RAGGED}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def affine(wl, c, seed):
    """c random affine rows: each touches three field rows and every control
    row, thresholds near the current values so some members violate."""
    rng = np.random.default_rng(seed)
    Gx = np.zeros((c, wl.n), np.float32)
    for r in range(c):
        Gx[r, rng.choice(wl.n, 3, replace=False)] = rng.standard_normal(3)
    Gu = rng.standard_normal((c, wl.l)).astype(np.float32)
    h = (0.05 * rng.standard_normal(c)).astype(np.float32)
    return W.Constraints(Gx, Gu, h, alpha=2.0, beta=20.0, sigma_z=0.01)


def spec_for(wl, kind):
    return W.u_box(wl.n, wl.l, 0.1) if kind == "box" else affine(wl, 5, 3)


def solver(wc, **kw):
    w, b = wc.flat_weights()
    return oic.Solver(oic.config_from_workload(wc, **kw), w, b, wc.B(), constraints=wc.cons)


def onet(wl):
    return oracle.Net(wl.n, wl.m, wl.l, wl.channels, wl.weights(), wl.B(), wl.residual_scale)


def ocons(spec):
    return oracle.Cons(spec.Gx, spec.Gu, spec.h, spec.alpha, spec.beta)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("kind", ["box", "affine"])
@pytest.mark.parametrize("full", [False, True])
def test_constrained_solve_matches_oracle(cuda_ok, name, kind, full):
    wl = CASES[name]
    wc = wl.with_(cons=spec_for(wl, kind))
    s = solver(wc, keep_full_history=full)
    assert s.noise_floats == wc.noise_floats()
    k = 1
    Xk = wl.X0()
    Up = np.zeros((wl.l, wl.m), np.float32)
    ur = np.full((wl.l, wl.m), 0.2, np.float32)           # outside the box
    xr, nz = wl.X_ref_window(k), wc.noise(k)
    U_hat = np.zeros((wl.H + 1, wl.l, wl.m), np.float32)
    X_hat = np.zeros((wl.H + 1, wl.n, wl.m), np.float32) if full else None
    s.oic_solve_host(Xk, Up, xr, ur, nz, U_hat, X_hat)
    xh = oracle.enks_solve(onet(wl), wl.N, wl.H, Xk, Up, xr, ur, nz, ocons(wc.cons))
    assert rel(U_hat, xh[:, wl.n:wl.n + wl.l]) <= TOL
    if full:
        assert rel(X_hat, xh[:, :wl.n]) <= TOL
    # the rows carry weight: without them the oracle's controls differ by far more
    plain = oracle.enks_solve(onet(wl), wl.N, wl.H, Xk, Up, xr, ur, wl.noise(k))
    assert rel(plain[:, wl.n:wl.n + wl.l], xh[:, wl.n:wl.n + wl.l]) > 100 * TOL
    s.close()


def _philox_steps(wc, steps, seed):
    s = solver(wc, noise_mode=oic.OIC_NOISE_PHILOX, seed=seed)
    xr_all = wc.X_ref_all(steps)
    ur = np.full((wc.l, wc.m), 0.2, np.float32)
    s.oic_reset_host(wc.X0(), wc.U_init())
    out = []
    for k in range(steps):
        Ua = np.zeros((wc.l, wc.m), np.float32)
        Xn = np.zeros((wc.n, wc.m), np.float32)
        s.oic_step_host(xr_all[k:k + wc.H + 1], ur, None, Ua, Xn)
        out.append((Ua, Xn))
    s.close()
    return out


@pytest.mark.parametrize("name", ["small_16", "tc_ragged"])
def test_constrained_philox_steps_match_oracle_and_eager(cuda_ok, name, monkeypatch):
    """Philox mode draws eps as a fifth noise segment; the step graph (with the
    constraint kernel in it) replays bit-identically to eager launches, and the
    closed loop follows the oracle fed the host restatement of the Philox
    noise."""
    wl = CASES[name]
    wc = wl.with_(cons=W.u_box(wl.n, wl.l, 0.1))
    steps, seed = 3, 4321
    graph = _philox_steps(wc, steps, seed)
    monkeypatch.setenv("OIC_NO_GRAPH", "1")
    eager = _philox_steps(wc, steps, seed)
    for (ga, gx), (ea, ex) in zip(graph, eager):
        assert np.array_equal(ga, ea) and np.array_equal(gx, ex)
    net, cons = onet(wl), ocons(wc.cons)
    xr_all = wl.X_ref_all(steps)
    ur = np.full((wl.l, wl.m), 0.2)
    X = wl.X0().astype(np.float64)
    Up = wl.U_init().astype(np.float64)
    for k in range(steps):
        nz = W.philox_noise(wc, solve=k, seed=seed)
        xh = oracle.enks_solve(net, wl.N, wl.H, X, Up, xr_all[k:k + wl.H + 1], ur, nz, cons)
        Uo = xh[0, wl.n:wl.n + wl.l]
        assert rel(graph[k][0], Uo) <= TOL
        X = oracle.cnn_step(net, X, Uo)
        Up = Uo
        assert rel(graph[k][1], X) <= TOL


def test_constrained_working_size_tensor_path(cuda_ok):
    """64 x 64 field, l = 8, the 2-32-32-1 CNN on the fused tensor-core kernel,
    the box adding 16 observed rows (p = 88); N and H reduced so the oracle
    finishes in seconds."""
    wl = W.working_64().with_(N=64, H=3)
    wc = wl.with_(cons=W.u_box(wl.n, wl.l, 0.1))
    s = solver(wc)
    k = 0
    Up = np.zeros((wl.l, wl.m), np.float32)
    ur = np.full((wl.l, wl.m), 0.2, np.float32)
    xr, nz = wl.X_ref_window(k), wc.noise(k)
    U_hat = np.zeros((wl.H + 1, wl.l, wl.m), np.float32)
    s.oic_solve_host(wl.X0(), Up, xr, ur, nz, U_hat)
    xh = oracle.enks_solve(onet(wl), wl.N, wl.H, wl.X0(), Up, xr, ur, nz, ocons(wc.cons))
    assert rel(U_hat, xh[:, wl.n:wl.n + wl.l]) <= TOL
    s.close()


def test_analyses_of_different_observation_counts_on_one_handle(cuda_ok):
    """One constrained handle alternates constrained solves (p = n + l + c
    observed rows: 42 here, Sigma^Y staged for the FP32 gain as 48 rows of 49)
    with a plain analysis through oic_enks_update (p = n + l = 36: 40 rows of
    41), so the staged copy of Sigma^Y changes layout from call to call over
    the same buffer.  Each result must match the oracle: a call may read only
    its own rows, whatever the previous call left behind."""
    import torch

    wl = MID
    wc = wl.with_(cons=affine(wl, 6, 3))
    s = solver(wc)
    Up = np.zeros((wl.l, wl.m), np.float32)
    ur = np.full((wl.l, wl.m), 0.2, np.float32)
    net, cons = onet(wl), ocons(wc.cons)

    def constrained(k):
        xr, nz = wl.X_ref_window(k), wc.noise(k)
        U_hat = np.zeros((wl.H + 1, wl.l, wl.m), np.float32)
        s.oic_solve_host(wl.X0(), Up, xr, ur, nz, U_hat)
        xh = oracle.enks_solve(net, wl.N, wl.H, wl.X0(), Up, xr, ur, nz, cons)
        assert rel(U_hat, xh[:, wl.n:wl.n + wl.l]) <= TOL

    def plain(seed):
        rng = np.random.default_rng(seed)
        R, p = 45, wl.n + wl.l
        E = (1.0 + 0.05 * rng.standard_normal((wl.N, R, wl.m))).astype(np.float32)
        obs = np.sort(rng.choice(R, size=p, replace=False))
        V = (0.02 * rng.standard_normal((wl.N, p, wl.m))).astype(np.float32)
        Ybar = (1.2 + 0.1 * rng.standard_normal((p, wl.m))).astype(np.float32)
        Ed = torch.from_numpy(E).cuda()
        s.oic_enks_update(Ed, obs, torch.from_numpy(V).cuda(), torch.from_numpy(Ybar).cuda())
        s.oic_sync()
        got = Ed.cpu().numpy()
        want = oracle.enks_analysis(E, E[:, obs, :] + V, Ybar)
        assert rel(got - E, want - E) <= TOL

    constrained(1)
    plain(11)
    constrained(2)
    plain(12)
    s.close()

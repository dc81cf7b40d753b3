"""Scheduling plans and the autotuner (oic_get_plan / oic_set_plan /
oic_autotune) on the GPU.

A plan changes how the kernels are laid out on the GPU, never what they
compute: CTA counts of the persistent CNN and member-update kernels leave
every result bit-identical; the member-split count of the covariance
products regroups FP32 partial sums, so results stay within the FP32 parity
bar of the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
import paper_2410_09663_b300 as oic
from paper_2410_09663_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-4


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def solver(wl, **kw):
    w, b = wl.flat_weights()
    return oic.Solver(oic.config_from_workload(wl, **kw), w, b, wl.B())


def onet(wl):
    return oracle.Net(wl.n, wl.m, wl.l, wl.channels, wl.weights(), wl.B(), wl.residual_scale)


def philox_steps(s, wl, steps):
    xr = wl.X_ref_all(steps)
    out = []
    for k in range(steps):
        Ua = np.zeros((wl.l, wl.m), np.float32)
        Xn = np.zeros((wl.n, wl.m), np.float32)
        s.oic_step_host(xr[k:k + wl.H + 1], wl.U_ref(), None, Ua, Xn)
        out.append((Ua, Xn))
    return out


FUSED = W.working_64().with_(N=32, H=3)
MIXED = W.Workload("plan_mixed_32", n=32, m=32, l=4, channels=[2, 64, 64, 64, 1], N=24, H=2, S=2, ref="blobs",
                   blob_sigma=3.0)


@pytest.mark.parametrize("name", ["fused", "mixed"])
def test_cta_counts_leave_results_bit_identical(cuda_ok, name):
    wl, prec = (FUSED, oic.OIC_PREC_FP32) if name == "fused" else (MIXED, oic.OIC_PREC_MIXED)
    runs = []
    for plan in ({}, {"cnn_ctas": 74, "update_ctas": 37}, {"cnn_ctas": 131, "update_ctas": 111}):
        s = solver(wl, noise_mode=oic.OIC_NOISE_PHILOX, seed=5, precision=prec)
        s.oic_set_plan(**plan)
        got, _ = s.oic_get_plan()
        for k, v in plan.items():
            assert got[k] == v
        s.oic_reset_host(wl.X0(), wl.U_init())
        runs.append(philox_steps(s, wl, 3))
        s.close()
    for other in runs[1:]:
        for (a0, x0), (a1, x1) in zip(runs[0], other):
            assert np.array_equal(a0, a1) and np.array_equal(x0, x1)


def test_split_counts_stay_within_the_fp32_bar(cuda_ok):
    wl = FUSED
    s = solver(wl)
    _, lim = s.oic_get_plan()
    Up = (0.01 * np.random.default_rng(3).standard_normal((wl.l, wl.m))).astype(np.float32)
    xr, ur, nz = wl.X_ref_window(1), wl.U_ref(), wl.noise(1)
    want = oracle.enks_solve(onet(wl), wl.N, wl.H, wl.X0(), Up, xr, ur, nz)[:, wl.n:wl.n + wl.l]
    for splits in sorted({1, 2, 3, max(1, lim["stats_splits"] // 2), lim["stats_splits"]}):
        s.oic_set_plan(stats_splits=splits)
        assert s.oic_get_plan()[0]["stats_splits"] == splits
        U_hat = np.zeros((wl.H + 1, wl.l, wl.m), np.float32)
        s.oic_solve_host(wl.X0(), Up, xr, ur, nz, U_hat)
        assert rel(U_hat, want) <= TOL, splits
    s.close()


def test_set_plan_rejects_values_outside_the_limits(cuda_ok):
    s = solver(FUSED)
    _, lim = s.oic_get_plan()
    for bad in ({"stats_splits": -1}, {"update_ctas": lim["update_ctas"] + 1}, {"cnn_ctas": lim["cnn_ctas"] + 1},
                {"stats_splits": lim["stats_splits"] + 1}):
        with pytest.raises(oic.OICError) as e:
            s.oic_set_plan(**bad)
        assert e.value.status == oic.OIC_EINVAL
    s.close()


def test_autotune_keeps_the_state_matches_the_oracle_and_caches(cuda_ok):
    """Tuning runs control steps of its own; afterwards the handle continues
    from the caller's state (plant, last control, solve index), so the next
    steps match the FP64 oracle fed the same Philox numbers.  A second handle
    of the same shape takes the plan from the cache without timing."""
    wl = W.small_16()
    seed = 77
    s = solver(wl, noise_mode=oic.OIC_NOISE_PHILOX, seed=seed)
    s.oic_reset_host(wl.X0(), wl.U_init())
    first = philox_steps(s, wl, 1)                      # solve index 0
    plan, ms_rule, ms_tuned = s.oic_autotune(reps=2, force=True)
    assert ms_rule > 0 and 0 < ms_tuned <= ms_rule
    _, lim = s.oic_get_plan()
    for k in plan:
        assert 1 <= plan[k] <= lim[k]
    xr_all = wl.X_ref_all(4)
    net = onet(wl)
    X = oracle.cnn_step(net, wl.X0(), first[0][0]).astype(np.float64)
    Up = first[0][0].astype(np.float64)
    for k in range(1, 3):                               # solve indices 1, 2 continue the stream
        Ua = np.zeros((wl.l, wl.m), np.float32)
        Xn = np.zeros((wl.n, wl.m), np.float32)
        s.oic_step_host(xr_all[k:k + wl.H + 1], wl.U_ref(), None, Ua, Xn)
        nz = W.philox_noise(wl, solve=k, seed=seed)
        Uo = oracle.enks_solve(net, wl.N, wl.H, X, Up, xr_all[k:k + wl.H + 1], wl.U_ref(), nz)[0, wl.n:wl.n + wl.l]
        assert rel(Ua, Uo) <= TOL
        X = oracle.cnn_step(net, X, Uo)
        Up = Uo
        assert rel(Xn, X) <= TOL
    s2 = solver(wl, noise_mode=oic.OIC_NOISE_PHILOX, seed=seed)
    s2.oic_reset_host(wl.X0(), wl.U_init())
    plan2, a, b = s2.oic_autotune(reps=2)
    assert plan2 == plan and a == -1.0 and b == -1.0
    s.close()
    s2.close()


def test_autotune_requires_a_plant(cuda_ok):
    s = solver(W.small_16(), noise_mode=oic.OIC_NOISE_PHILOX)
    with pytest.raises(oic.OICError) as e:
        s.oic_autotune()
    assert e.value.status == oic.OIC_ESTATE
    s.close()


def test_batch_autotune_results_equal_each_problem_alone_with_its_plan(cuda_ok):
    """oic_batch_autotune picks plans by timing whole batch steps; afterwards
    each problem in the batch gives, bit for bit, what the same problem
    stepped alone with the same plan gives, and the state it had before the
    tuning is kept (the first tuned batch step is solve index 0)."""
    import torch
    wls = [W.small_16(), W.working_64().with_(N=32, H=3, seed=11), MIXED.with_(seed=5)]
    precs = [oic.OIC_PREC_FP32, oic.OIC_PREC_FP32, oic.OIC_PREC_MIXED]
    solvers = []
    for w, pr in zip(wls, precs):
        s = solver(w, noise_mode=oic.OIC_NOISE_PHILOX, precision=pr)
        s.oic_reset_host(w.X0(), w.U_init())
        solvers.append(s)
    batch = oic.Batch(solvers)
    ms_rule, ms_tuned = batch.autotune(reps=2)
    assert ms_rule > 0 and 0 < ms_tuned <= ms_rule
    plans = [s.oic_get_plan()[0] for s in solvers]
    steps = 2
    slots = [s.oic_io_slots() for s in solvers]
    got = []
    for k in range(steps):
        for w, (xr, ur, _, _) in zip(wls, slots):
            xr.copy_(torch.from_numpy(w.X_ref_all(steps)[k:k + w.H + 1]).to(xr.device))
            ur.copy_(torch.from_numpy(w.U_ref()).to(ur.device))
        batch.step()
        batch.sync()
        got.append([(sua.cpu().numpy(), sxn.cpu().numpy()) for (_, _, sua, sxn) in slots])
    batch.close()
    for i, (w, pr, plan) in enumerate(zip(wls, precs, plans)):
        s = solver(w, noise_mode=oic.OIC_NOISE_PHILOX, precision=pr)
        s.oic_set_plan(**plan)
        s.oic_reset_host(w.X0(), w.U_init())
        alone = philox_steps(s, w, steps)
        for k in range(steps):
            assert np.array_equal(got[k][i][0], alone[k][0])
            assert np.array_equal(got[k][i][1], alone[k][1])
        s.close()

"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerance: relative L2 error <= 1e-4 on ensemble means and controls for the
FP32 path (the bar the method's FP32 configuration is held to); the CNN alone
is held to 1e-5 per element relative to the field's scale (a few FP32 ulps
through K = 9 * C_in term dot products).
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


def onet(wl):
    return oracle.Net(wl.n, wl.m, wl.l, wl.channels, wl.weights(), wl.B(), wl.residual_scale)


def solver(wl, **kw):
    w, b = wl.flat_weights()
    return oic.Solver(oic.config_from_workload(wl, **kw), w, b, wl.B())


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


RAGGED = W.Workload("ragged_20x24", n=20, m=24, l=3, channels=[2, 6, 1], N=19, H=3, S=4, ref="blobs",
                    blob_sigma=3.0)
MID = W.Workload("mid_32x48", n=32, m=48, l=4, channels=[2, 16, 16, 1], N=64, H=4, S=3, ref="blobs",
                 blob_sigma=4.0)
# hidden 32 -> 32 layer on the tensor cores; m = 32 puts 4 members in a
# 128-pixel tile and N = 13 leaves the last tile with one member
TC_RAGGED = W.Workload("tc_24x32", n=24, m=32, l=4, channels=[2, 32, 32, 1], N=13, H=3, S=3,
                       ref="blobs", blob_sigma=4.0)
CASES = {"small_16": W.small_16(), "ragged": RAGGED, "mid": MID, "tc_ragged": TC_RAGGED}


def test_tensor_core_selftest(cuda_ok):
    s = solver(W.small_16())
    st, res = s.oic_selftest()
    assert st == oic.OIC_OK and res[0] == 0, res


@pytest.mark.parametrize("name", ["small_16", "ragged", "mid", "tc_ragged", "working_64"])
def test_cnn_forward_matches_oracle(cuda_ok, name):
    wl = CASES[name] if name in CASES else W.working_64()
    batch = min(wl.N, 6)
    rng = np.random.default_rng(5)
    X = (wl.X0()[None] + 0.3 * rng.standard_normal((batch, wl.n, wl.m))).astype(np.float32)
    U = (0.5 * rng.standard_normal((batch, wl.l, wl.m))).astype(np.float32)
    s = solver(wl)
    Xd, Ud = dev(X), dev(U)
    out = dev(np.zeros_like(X))
    s.oic_cnn_forward(Xd, Ud, out)
    s.oic_sync()
    got = out.cpu().numpy()
    want = oracle.cnn_step(onet(wl), X, U)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()


def test_cnn_forward_rejects_overlapping_output(cuda_ok):
    """X_next overlapping X is refused before any launch (halo rows of X are
    read by neighbouring tiles while others write X_next)."""
    wl = CASES["small_16"]
    s = solver(wl)
    X = dev(np.zeros((2, wl.n, wl.m), np.float32))
    U = dev(np.zeros((2, wl.l, wl.m), np.float32))
    with pytest.raises(oic.OICError) as e:
        s.oic_cnn_forward(X, U, X)
    assert e.value.status == oic.OIC_EINVAL
    with pytest.raises(oic.OICError) as e:
        shifted = X.view(-1)[wl.m: wl.m + wl.n * wl.m].view(1, wl.n, wl.m)   # one image row into X[0]
        s.oic_cnn_forward(X[:1], U[:1], shifted)
    assert e.value.status == oic.OIC_EINVAL


@pytest.mark.parametrize("name", ["small_16", "ragged", "mid", "tc_ragged"])
@pytest.mark.parametrize("full", [False, True])
def test_solve_matches_oracle(cuda_ok, name, full):
    wl = CASES[name]
    s = solver(wl, keep_full_history=full)
    k = 2
    Xk = wl.X0()
    Up = (0.01 * np.random.default_rng(7).standard_normal((wl.l, wl.m))).astype(np.float32)
    xr, ur, nz = wl.X_ref_window(k), wl.U_ref(), wl.noise(k)
    U_hat = np.zeros((wl.H + 1, wl.l, wl.m), np.float32)
    X_hat = np.zeros((wl.H + 1, wl.n, wl.m), np.float32) if full else None
    s.oic_solve_host(Xk, Up, xr, ur, nz, U_hat, X_hat)
    xh = oracle.enks_solve(onet(wl), wl.N, wl.H, Xk, Up, xr, ur, nz)
    assert rel(U_hat, xh[:, wl.n:wl.n + wl.l]) <= TOL
    if full:
        assert rel(X_hat, xh[:, :wl.n]) <= TOL


def test_device_and_host_entry_points_agree(cuda_ok):
    wl = MID
    s = solver(wl)
    Xk, Up = wl.X0(), wl.U_init()
    xr, ur, nz = wl.X_ref_window(0), wl.U_ref(), wl.noise(0)
    U_host = np.zeros((wl.H + 1, wl.l, wl.m), np.float32)
    s.oic_solve_host(Xk, Up, xr, ur, nz, U_host)
    U_dev = dev(np.zeros_like(U_host))
    s.oic_solve(dev(Xk), dev(Up), dev(xr), dev(ur), dev(nz), U_dev)
    s.oic_sync()
    np.testing.assert_array_equal(U_dev.cpu().numpy(), U_host)


@pytest.mark.parametrize("name", ["small_16", "ragged"])
def test_closed_loop_matches_oracle(cuda_ok, name):
    wl = CASES[name]
    S = wl.S
    s = solver(wl)
    xr_all = wl.X_ref_all(S)
    s.oic_reset_host(wl.X0(), wl.U_init())
    Ut = np.zeros((S, wl.l, wl.m), np.float32)
    Xt = np.zeros((S + 1, wl.n, wl.m), np.float32)
    Xt[0] = wl.X0()
    for k in range(S):
        s.oic_step_host(xr_all[k:k + wl.H + 1], wl.U_ref(), wl.noise(k), Ut[k], Xt[k + 1])
    Xo, Uo, _ = oracle.run(onet(wl), wl.N, wl.H, S, wl.X0(), wl.U_init(), xr_all, wl.U_ref(),
                           wl.noise_all(S))
    assert rel(Ut, Uo) <= TOL
    assert rel(Xt, Xo) <= TOL
    jg = oracle.closed_loop_cost(Xt, Ut, xr_all, wl.U_ref(), wl.U_init(), wl.sigma_vx, wl.sigma_vu,
                                 wl.sigma_w)
    jo = oracle.closed_loop_cost(Xo, Uo, xr_all, wl.U_ref(), wl.U_init(), wl.sigma_vx, wl.sigma_vu,
                                 wl.sigma_w)
    assert abs(jg - jo) <= 1e-4 * abs(jo)


def test_philox_mode_matches_oracle_fed_host_philox(cuda_ok):
    wl = W.small_16()
    s = solver(wl, noise_mode=oic.OIC_NOISE_PHILOX, seed=1234)
    net = onet(wl)
    xr_all = wl.X_ref_all(3)
    s.oic_reset_host(wl.X0(), wl.U_init())
    X = wl.X0().astype(np.float64)
    Up = wl.U_init().astype(np.float64)
    for k in range(3):
        Ua = np.zeros((wl.l, wl.m), np.float32)
        Xn = np.zeros((wl.n, wl.m), np.float32)
        s.oic_step_host(xr_all[k:k + wl.H + 1], wl.U_ref(), None, Ua, Xn)
        nz = W.philox_noise(wl, solve=k, seed=1234)
        xh = oracle.enks_solve(net, wl.N, wl.H, X, Up, xr_all[k:k + wl.H + 1], wl.U_ref(), nz)
        Uo = xh[0, wl.n:wl.n + wl.l]
        assert rel(Ua, Uo) <= TOL
        X = oracle.cnn_step(net, X, Uo)
        Up = Uo
        assert rel(Xn, X) <= TOL


def _philox_steps(wl, steps, profile=None, sample=None):
    s = solver(wl, noise_mode=oic.OIC_NOISE_PHILOX, seed=99)
    xr_all = wl.X_ref_all(steps)
    s.oic_reset_host(wl.X0(), wl.U_init())
    if profile is not None:
        s.oic_profile_begin(stages=profile, max_launches=4096)
        if sample is not None:
            s.oic_profile_sample(*sample)
    out = []
    for k in range(steps):
        Ua = np.zeros((wl.l, wl.m), np.float32)
        Xn = np.zeros((wl.n, wl.m), np.float32)
        s.oic_step_host(xr_all[k:k + wl.H + 1], wl.U_ref(), None, Ua, Xn)
        out.append((Ua, Xn))
    prof = s.oic_profile_end() if profile is not None else None
    s.close()
    return out, prof


@pytest.mark.parametrize("eager", [False, True])
def test_profile_sampling_brackets_only_the_chosen_launches(cuda_ok, monkeypatch, eager):
    """oic_profile_sample(every, phase): of a stage's launches in one solve
    (counted from 0), only those with index % every == phase carry events, in
    the step graph and in eager launches alike, and the results stay
    bit-identical to unprofiled steps.  The gain runs once per analysis, H
    times per solve."""
    wl = W.small_16()
    if eager:
        monkeypatch.setenv("OIC_NO_GRAPH", "1")
    base, _ = _philox_steps(wl, 3)
    one, p1 = _philox_steps(wl, 3, profile=["gain"], sample=(wl.H, wl.H // 2))
    two, p2 = _philox_steps(wl, 3, profile=["gain"], sample=(2, 1))
    _, pall = _philox_steps(wl, 3, profile=["gain"])
    assert p1["gain"][1] == 3 and p1["gain"][0] > 0
    assert p2["gain"][1] == 3 * (wl.H // 2)                # indices 1, 3, ... < H
    assert pall["gain"][1] == 3 * wl.H
    for (ba, bx), (oa, ox), (ta, tx) in zip(base, one, two):
        assert np.array_equal(ba, oa) and np.array_equal(bx, ox)
        assert np.array_equal(ba, ta) and np.array_equal(bx, tx)


def test_profile_sampling_rejects_bad_arguments(cuda_ok):
    wl = W.small_16()
    s = solver(wl, noise_mode=oic.OIC_NOISE_PHILOX, seed=99)
    with pytest.raises(RuntimeError):
        s.oic_profile_sample(2, 0)                            # no profile open
    s.oic_profile_begin(stages=["gain"], max_launches=16)
    for every, phase in ((0, 0), (3, 3), (2, -1)):
        with pytest.raises(RuntimeError):
            s.oic_profile_sample(every, phase)
    s.oic_profile_sample(3, 2)
    s.oic_profile_end()
    s.close()


@pytest.mark.parametrize("name", ["small_16", "working_64_n32"])
def test_step_graph_replays_match_eager_launches(cuda_ok, name, monkeypatch):
    """A control step replayed from its CUDA graph (plain, and with the
    profiling event nodes re-pointed before each replay) gives bit-identical
    controls and states to the same step launched kernel by kernel; the
    device-side solve index advances the Philox stream on every replay."""
    wl = W.small_16() if name == "small_16" else W.working_64().with_(N=32, H=3)
    graph, _ = _philox_steps(wl, 3)
    profiled, prof = _philox_steps(wl, 3, profile=["cov", "gain"])
    monkeypatch.setenv("OIC_NO_GRAPH", "1")
    eager, _ = _philox_steps(wl, 3)
    for (ga, gx), (pa, px), (ea, ex) in zip(graph, profiled, eager):
        assert np.array_equal(ga, ea) and np.array_equal(gx, ex)
        assert np.array_equal(pa, ea) and np.array_equal(px, ex)
    assert not np.array_equal(graph[0][0], graph[1][0])    # fresh noise each step
    assert prof["cov"][1] == 3 * wl.H and prof["gain"][1] == 3 * wl.H
    assert prof["cov"][0] > 0 and prof["gain"][0] > 0
    assert set(prof) == {"cov", "gain"}


def _device_noise_steps(wl, steps, precision, cons=None):
    w, b = wl.flat_weights()
    s = oic.Solver(oic.config_from_workload(wl, noise_mode=oic.OIC_NOISE_PHILOX, seed=31, precision=precision),
                   w, b, wl.B(), constraints=cons)
    s.oic_reset_host(wl.X0(), wl.U_init())
    xr_all = wl.X_ref_all(steps)
    out = []
    for k in range(steps):
        Ua = np.zeros((wl.l, wl.m), np.float32)
        Xn = np.zeros((wl.n, wl.m), np.float32)
        s.oic_step_host(xr_all[k:k + wl.H + 1], wl.U_ref(), None, Ua, Xn)
        out.append((Ua, Xn))
    s.close()
    return out


@pytest.mark.parametrize("case", ["fused", "mixed", "per_layer", "constrained"])
def test_noise_drawn_in_place_equals_the_noise_buffer(cuda_ok, case, monkeypatch):
    """Device-noise mode: the kernels that consume the random numbers draw
    them in place from the Philox stream; with OIC_NOISE_BUFFER the noise
    kernel writes the stream to the buffer first and they read it.  The two
    give bit-identical controls and states, step after step."""
    cons = None
    prec = oic.OIC_PREC_FP32
    if case == "fused":
        wl = W.working_64().with_(N=32, H=3)
    elif case == "mixed":
        wl, prec = MIXED_CASES["m32_c64"].with_(N=24, H=3, S=3), oic.OIC_PREC_MIXED
    elif case == "per_layer":
        wl = MID
    else:
        wl = W.small_16()
        cons = W.u_box(wl.n, wl.l, 0.05)
    drawn = _device_noise_steps(wl, 3, prec, cons)
    monkeypatch.setenv("OIC_NOISE_BUFFER", "1")
    buffered = _device_noise_steps(wl, 3, prec, cons)
    for (a0, x0), (a1, x1) in zip(drawn, buffered):
        assert np.array_equal(a0, a1) and np.array_equal(x0, x1)
    assert not np.array_equal(drawn[0][0], drawn[1][0])


@pytest.mark.parametrize("precision", [oic.OIC_PREC_FP32, oic.OIC_PREC_MIXED])
def test_enks_update_matches_oracle(cuda_ok, precision):
    """FP32 mode: FP32 gain by elimination; mixed mode: FP64 mean correction,
    FP64 Cholesky gain (the MID CNN has 16 channels, outside the BF16 path,
    so only the analysis differs)."""
    wl = MID
    s = solver(wl, precision=precision)
    rng = np.random.default_rng(9)
    R = 45
    p = wl.p
    assert p < R <= s.max_rows
    E = (1.0 + 0.05 * rng.standard_normal((wl.N, R, wl.m))).astype(np.float32)
    obs = np.sort(rng.choice(R, size=p, replace=False))
    V = (0.02 * rng.standard_normal((wl.N, p, wl.m))).astype(np.float32)
    Ybar = (1.2 + 0.1 * rng.standard_normal((p, wl.m))).astype(np.float32)
    Ed = dev(E)
    s.oic_enks_update(Ed, obs, dev(V), dev(Ybar))
    s.oic_sync()
    got = Ed.cpu().numpy()
    want = oracle.enks_analysis(E, E[:, obs, :] + V, Ybar)
    assert rel(got - E, want - E) <= TOL
    assert rel(got.mean(0), want.mean(0)) <= TOL


@pytest.mark.parametrize("precision", [oic.OIC_PREC_FP32, oic.OIC_PREC_MIXED])
def test_not_positive_definite_is_reported_and_skipped(cuda_ok, precision):
    wl = MID
    s = solver(wl, precision=precision)
    R = wl.p
    E = np.ones((wl.N, R, wl.m), np.float32)        # identical members, V = 0: Sigma^Y = 0
    V = np.zeros((wl.N, wl.p, wl.m), np.float32)
    Ed = dev(E)
    s.oic_enks_update(Ed, np.arange(wl.p), dev(V), dev(np.zeros((wl.p, wl.m), np.float32)))
    assert s.oic_sync_status() == oic.OIC_ENOTSPD
    np.testing.assert_array_equal(Ed.cpu().numpy(), E)
    assert s.oic_sync_status() == oic.OIC_OK       # status is cleared once read


@pytest.mark.slow
def test_working_size_one_control_step(cuda_ok):
    """Full-size bench workload (64 x 64, N = 256, H = 10, CNN 2-32-32-1), one
    control step through the same entry point the benchmark times."""
    wl = W.working_64()
    s = solver(wl)
    xr_all = wl.X_ref_all(1)
    s.oic_reset_host(wl.X0(), wl.U_init())
    Ua = np.zeros((wl.l, wl.m), np.float32)
    Xn = np.zeros((wl.n, wl.m), np.float32)
    s.oic_step_host(xr_all[:wl.H + 1], wl.U_ref(), wl.noise(0), Ua, Xn)
    Xo, Uo, _ = oracle.run(onet(wl), wl.N, wl.H, 1, wl.X0(), wl.U_init(), xr_all, wl.U_ref(),
                           wl.noise_all(1))
    assert rel(Ua, Uo[0]) <= TOL
    assert rel(Xn, Xo[1]) <= TOL


def test_large_128_cnn_sampled_members(cuda_ok):
    """128 x 128 field, CNN 2-64-64-64-1 at full size: run all N = 1024 members
    through the rollout kernels and check a sample of members one by one."""
    import torch
    wl = W.large_128()
    s = solver(wl)
    rng = np.random.default_rng(3)
    X = torch.from_numpy(wl.X0()).cuda()[None].repeat(wl.N, 1, 1)
    X += 0.05 * torch.randn_like(X)
    U = 0.3 * torch.randn(wl.N, wl.l, wl.m, device="cuda")
    out = torch.zeros_like(X)
    s.oic_cnn_forward(X, U, out)
    s.oic_sync()
    idx = rng.choice(wl.N, size=3, replace=False)
    want = oracle.cnn_step(onet(wl), X[idx].cpu().numpy(), U[idx].cpu().numpy())
    got = out[idx].cpu().numpy()
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()


@pytest.mark.parametrize("name", ["tc_ragged", "working_64"])
def test_cnn_per_layer_tensor_path_matches_oracle(cuda_ok, name, monkeypatch):
    """The per-layer tensor-core path (used for hidden stacks other than one
    32 -> 32 layer) stays exact when the fused kernel is switched off."""
    monkeypatch.setenv("OIC_NO_FUSED_CNN", "1")
    wl = CASES[name] if name in CASES else W.working_64()
    batch = min(wl.N, 6)
    rng = np.random.default_rng(6)
    X = (wl.X0()[None] + 0.3 * rng.standard_normal((batch, wl.n, wl.m))).astype(np.float32)
    U = (0.5 * rng.standard_normal((batch, wl.l, wl.m))).astype(np.float32)
    s = solver(wl)
    out = dev(np.zeros_like(X))
    s.oic_cnn_forward(dev(X), dev(U), out)
    s.oic_sync()
    want = oracle.cnn_step(onet(wl), X, U)
    assert np.abs(out.cpu().numpy() - want).max() <= 1e-5 * np.abs(want).max()


MIXED_CASES = {
    "m16_c32": W.Workload("mixed_16x16_c32", n=16, m=16, l=4, channels=[2, 32, 32, 1], N=40, H=2, S=2, ref="zero"),
    "m32_c64": W.Workload("mixed_32x32_c64", n=32, m=32, l=4, channels=[2, 64, 64, 64, 1], N=12, H=2, S=2,
                          ref="zero"),
    "m64_c64": W.Workload("mixed_64x64_c64", n=64, m=64, l=8, channels=[2, 64, 64, 1], N=6, H=2, S=2, ref="zero"),
    "m128_c64": W.Workload("mixed_128x128_c64", n=128, m=128, l=16, channels=[2, 64, 64, 64, 1], N=3, H=2, S=2,
                           ref="zero"),
    "m96_c32": W.Workload("mixed_96x96_c32", n=96, m=96, l=12, channels=[2, 32, 32, 1], N=5, H=2, S=2, ref="zero"),
}


@pytest.mark.parametrize("name", list(MIXED_CASES))
def test_mixed_precision_cnn_within_bf16_bound(cuda_ok, name):
    """Mixed mode: BF16 operands, FP32 accumulation and residual.  Every
    operand is rounded once to 8 significant bits (unit roundoff u = 2^-9), so
    the CNN increment X_next - X carries a relative error of a few u; the
    bound is 4u in relative L2 and 8u in max norm of the increment."""
    wl = MIXED_CASES[name]
    s = solver(wl, precision=oic.OIC_PREC_MIXED)
    rng = np.random.default_rng(5)
    X = (wl.X0()[None] + 0.3 * rng.standard_normal((wl.N, wl.n, wl.m))).astype(np.float32)
    U = (0.5 * rng.standard_normal((wl.N, wl.l, wl.m))).astype(np.float32)
    out = dev(np.zeros_like(X))
    s.oic_cnn_forward(dev(X), dev(U), out)
    s.oic_sync()
    got = out.cpu().numpy().astype(np.float64)
    want = oracle.cnn_step(onet(wl), X, U)
    inc = want - X
    u = 2.0 ** -9
    assert np.linalg.norm(got - want) <= 4 * u * np.linalg.norm(inc)
    assert np.abs(got - want).max() <= 8 * u * np.abs(inc).max()


MIXED_LOOP = {
    "m16_c32": W.Workload("mixed_loop_16", n=16, m=16, l=4, channels=[2, 32, 32, 1], N=32, H=3, S=6, ref="zero"),
    "m32_c64": W.Workload("mixed_loop_32", n=32, m=32, l=4, channels=[2, 64, 64, 64, 1], N=32, H=3, S=4,
                          ref="blobs", blob_sigma=3.0),
}


@pytest.mark.parametrize("name", list(MIXED_LOOP))
def test_mixed_precision_closed_loop_cost_within_half_percent(cuda_ok, name):
    """Mixed mode (BF16 CNN, FP32 covariances, FP64 mean correction and
    gain) against the FP64 oracle fed the same noise: the closed-loop cost J
    within 0.5%, the applied controls within 4u of BF16 (u = 2^-9) in
    relative L2, the states within 1e-3."""
    wl = MIXED_LOOP[name]
    S = wl.S
    s = solver(wl, precision=oic.OIC_PREC_MIXED)
    xr_all = wl.X_ref_all(S)
    s.oic_reset_host(wl.X0(), wl.U_init())
    Ut = np.zeros((S, wl.l, wl.m), np.float32)
    Xt = np.zeros((S + 1, wl.n, wl.m), np.float32)
    Xt[0] = wl.X0()
    for k in range(S):
        s.oic_step_host(xr_all[k:k + wl.H + 1], wl.U_ref(), wl.noise(k), Ut[k], Xt[k + 1])
    Xo, Uo, _ = oracle.run(onet(wl), wl.N, wl.H, S, wl.X0(), wl.U_init(), xr_all, wl.U_ref(),
                           wl.noise_all(S))
    jg = oracle.closed_loop_cost(Xt, Ut, xr_all, wl.U_ref(), wl.U_init(), wl.sigma_vx, wl.sigma_vu,
                                 wl.sigma_w)
    jo = oracle.closed_loop_cost(Xo, Uo, xr_all, wl.U_ref(), wl.U_init(), wl.sigma_vx, wl.sigma_vu,
                                 wl.sigma_w)
    assert abs(jg - jo) <= 5e-3 * abs(jo)
    assert rel(Ut, Uo) <= 4 * 2.0 ** -9
    assert rel(Xt, Xo) <= 1e-3


def _steps_alone(wl, steps, precision):
    s = solver(wl, noise_mode=oic.OIC_NOISE_PHILOX, precision=precision)
    s.oic_reset_host(wl.X0(), wl.U_init())
    xr_all = wl.X_ref_all(steps)
    out = []
    for k in range(steps):
        Ua = np.zeros((wl.l, wl.m), np.float32)
        Xn = np.zeros((wl.n, wl.m), np.float32)
        s.oic_step_host(xr_all[k:k + wl.H + 1], wl.U_ref(), None, Ua, Xn)
        out.append((Ua, Xn))
    s.close()
    return out


def test_batched_uneven_problems_equal_each_problem_alone(cuda_ok):
    """Problems of different grid, ensemble and horizon sizes (one of them in
    the mixed-precision mode) stepped together as one batch graph give the
    same controls and states, bit for bit, as each problem stepped alone."""
    import torch
    wls = [(W.small_16(), oic.OIC_PREC_FP32),
           (W.small_16().with_(N=48, H=3, seed=7), oic.OIC_PREC_FP32),
           (W.working_64().with_(N=32, H=3, seed=11), oic.OIC_PREC_FP32),
           (MIXED_CASES["m32_c64"].with_(seed=5), oic.OIC_PREC_MIXED)]
    steps = 3
    alone = [_steps_alone(w, steps, pr) for w, pr in wls]
    solvers = []
    for w, pr in wls:
        s = solver(w, noise_mode=oic.OIC_NOISE_PHILOX, precision=pr)
        s.oic_reset_host(w.X0(), w.U_init())
        solvers.append(s)
    batch = oic.Batch(solvers)
    slots = [s.oic_io_slots() for s in solvers]
    for k in range(steps):
        for (w, _), (xr, ur, _, _) in zip(wls, slots):
            xr.copy_(torch.from_numpy(w.X_ref_all(steps)[k:k + w.H + 1]).to(xr.device))
            ur.copy_(torch.from_numpy(w.U_ref()).to(ur.device))
        batch.step()
        batch.sync()
        for (ua, xn), (_, _, sua, sxn) in zip([a[k] for a in alone], slots):
            assert np.array_equal(sua.cpu().numpy(), ua)
            assert np.array_equal(sxn.cpu().numpy(), xn)
    batch.close()


def test_served_results_equal_each_problem_alone_with_evictions(cuda_ok):
    """The serving loop (continuous batching, admission by HBM footprint)
    under a budget that fits one problem at a time: requests of three
    problems arrive interleaved, so problems are evicted (state to the host)
    and re-admitted between their steps; every applied control equals, bit
    for bit, the same problem stepped alone and uninterrupted."""
    from paper_2410_09663_b300 import serving
    wls = [W.small_16(), W.small_16().with_(N=48, H=3, seed=7), W.small_16().with_(N=24, H=4, seed=9)]
    steps = 3
    alone = [_steps_alone(w, steps, oic.OIC_PREC_FP32) for w in wls]
    srv = serving.Server("cuda", budget_bytes=1, precision=oic.OIC_PREC_FP32, keep_outputs=True)
    for pid, w in enumerate(wls):
        srv.add(pid, w, steps_max=steps)
    srv.budget = max(p.bytes for p in srv.problems.values())
    arrivals = [(0.001 * i, i % 3) for i in range(3 * steps)]
    rec, outs, _ = srv.run(arrivals)
    for i, (t, pid) in enumerate(arrivals):
        k = rec[i][1]
        assert k == i // 3
        assert np.array_equal(outs[i], alone[pid][k][0])
    assert sum(p.evictions for p in srv.problems.values()) >= 2


def test_served_results_in_the_mix_equal_each_problem_alone(cuda_ok):
    """Continuous batching with every problem resident: requests of four
    problems of different grid, ensemble and horizon sizes arrive within a
    millisecond of each other, so steps of different problems are on
    the GPU at the same time (their CUDA-event intervals on the device
    overlap); every applied control equals, bit for bit, the same problem
    stepped alone, and nothing is evicted."""
    from paper_2410_09663_b300 import serving
    wls = [W.small_16(), W.small_16().with_(N=48, H=3, seed=7), W.working_64().with_(N=32, H=3, seed=11),
           W.small_16().with_(N=24, H=4, seed=9)]
    steps = 3
    alone = [_steps_alone(w, steps, oic.OIC_PREC_FP32) for w in wls]
    srv = serving.Server("cuda", budget_bytes=1, precision=oic.OIC_PREC_FP32, keep_outputs=True)
    for pid, w in enumerate(wls):
        srv.add(pid, w, steps_max=steps)
    srv.budget = sum(p.bytes for p in srv.problems.values())
    arrivals = [(0.0001 * i, i % len(wls)) for i in range(len(wls) * steps)]
    rec, outs, _ = srv.run(arrivals)
    for i, (t, pid) in enumerate(arrivals):
        k = rec[i][1]
        assert k == i // len(wls)
        assert np.array_equal(outs[i], alone[pid][k][0])
    assert sum(p.evictions for p in srv.problems.values()) == 0
    iv = srv.device_intervals
    overlapping = [(i, j) for i in range(len(iv)) for j in range(i + 1, len(iv))
                   if arrivals[i][1] != arrivals[j][1] and iv[i][0] < iv[j][1] and iv[j][0] < iv[i][1]]
    assert overlapping, iv
    assert serving.max_overlap(iv) >= 2


@pytest.mark.parametrize("l,mu,m", [(4, 1, 16), (8, 3, 64), (16, 8, 128), (5, 7, 24)])
def test_narrow_control_transform_matches_oracle(cuda_ok, l, mu, m):
    """U = u T and u = U T^T (T T^T)^{-1} against the FP64 oracle (expand:
    FP32 dot products of mu terms; reduce: FP64 inside, float32 out)."""
    rng = np.random.default_rng(l * 100 + mu)
    T = rng.standard_normal((mu, m)).astype(np.float32)
    u = rng.standard_normal((l, mu)).astype(np.float32)
    U = rng.standard_normal((l, m)).astype(np.float32)
    Ud = dev(np.zeros((l, m)))
    oic.oic_control_expand(dev(u), dev(T), Ud)
    want = oracle.control_expand(u, T)
    assert np.abs(Ud.cpu().numpy() - want).max() <= 1e-6 * max(1.0, np.abs(want).max()) * mu
    ud = dev(np.zeros((l, mu)))
    oic.oic_control_reduce(dev(U), dev(T), ud)
    want = oracle.control_reduce(U, T)
    assert np.abs(ud.cpu().numpy() - want).max() <= 2 ** -23 * np.abs(want).max() * 4
    ones = dev(np.ones((1, m)))
    u1 = dev(np.zeros((l, 1)))
    oic.oic_control_reduce(dev(U), ones, u1)
    np.testing.assert_allclose(u1.cpu().numpy()[:, 0], U.astype(np.float64).mean(axis=1), rtol=1e-6, atol=1e-7)


def test_narrow_control_reduce_reports_rank_deficient_transform(cuda_ok):
    T = np.array([[1.0, 2.0, 3.0, 4.0], [2.0, 4.0, 6.0, 8.0]], np.float32)
    u = dev(np.zeros((3, 2)))
    with pytest.raises(oic.OICError) as e:
        oic.oic_control_reduce(dev(np.ones((3, 4))), dev(T), u)
    assert e.value.status == oic.OIC_ENOTSPD


# ------------------------------------------------------------ edge cases
EDGE = {
    # the smallest ensemble (N = 2: the pooled sample covariance has (N-1) m = 16
    # samples for p = 5 rows), one assimilation, one control row
    "min_ensemble": W.Workload("edge_N2_H1", n=4, m=16, l=1, channels=[2, 32, 32, 1], N=2, H=1, S=2,
                               ref="blobs", blob_sigma=1.5),
    # the largest observation stack the FP32 path takes (p = n + l = 144)
    "max_p": W.Workload("edge_p144", n=128, m=16, l=16, channels=[2, 32, 32, 1], N=24, H=2, S=2, ref="blobs",
                        blob_sigma=8.0),
    # the widest grid (m = 128: one member per 128-position tile)
    "max_m": W.Workload("edge_m128", n=12, m=128, l=4, channels=[2, 32, 32, 1], N=6, H=2, S=2, ref="blobs",
                        blob_sigma=6.0),
}


@pytest.mark.parametrize("name", list(EDGE))
@pytest.mark.parametrize("full", [False, True])
def test_edge_case_solve_matches_oracle(cuda_ok, name, full):
    wl = EDGE[name]
    s = solver(wl, keep_full_history=full)
    Up = (0.01 * np.random.default_rng(9).standard_normal((wl.l, wl.m))).astype(np.float32)
    xr, ur, nz = wl.X_ref_window(1), wl.U_ref(), wl.noise(1)
    U_hat = np.zeros((wl.H + 1, wl.l, wl.m), np.float32)
    X_hat = np.zeros((wl.H + 1, wl.n, wl.m), np.float32) if full else None
    s.oic_solve_host(wl.X0(), Up, xr, ur, nz, U_hat, X_hat)
    xh = oracle.enks_solve(onet(wl), wl.N, wl.H, wl.X0(), Up, xr, ur, nz)
    assert rel(U_hat, xh[:, wl.n:wl.n + wl.l]) <= TOL
    if full:
        assert rel(X_hat, xh[:, :wl.n]) <= TOL
    s.close()


# ------------------------------------------- mixed precision at the 128 x 128 sizes
# The BF16 kernels hand each CTA a contiguous range of (member group, image
# row) passes, total / (number of SMs).  The cases below give every CTA tens
# of passes, so the 8-slot TMEM accumulator ring, the row-mod-8 barrier
# phases and the issue-ahead window wrap many times; the FP64 cluster gain
# sees p = 144 = 18 panels of 8 rows on 8 CTAs (block-cyclic, wrapping twice).
C2_CNN = {
    # first pair fused + last pair fused: 64 members x 128 rows = 8192 passes
    "m128_c64_N64": W.large_128().with_(N=64),
    # five layers: first pair, one per-layer 64 -> 64 kernel, last pair;
    # two members per tile, 64 groups x 64 rows = 4096 passes
    "m64_c64x4_N128": W.Workload("mixed_64x64_c64x4", n=64, m=64, l=8, channels=[2, 64, 64, 64, 64, 1], N=128,
                                 H=2, S=2, ref="blobs", blob_sigma=6.0),
    # three layers: input kernel, per-layer first layer, last pair; 8192 passes
    "m64_c64_N256": W.Workload("mixed_64x64_c64", n=64, m=64, l=8, channels=[2, 64, 64, 1], N=256, H=2, S=2,
                               ref="blobs", blob_sigma=6.0),
    # 32 channels, one member per 128-position tile (96 does not divide 128)
    "m96_c32_N64": W.Workload("mixed_96x96_c32_N64", n=96, m=96, l=12, channels=[2, 32, 32, 32, 1], N=64, H=2,
                              S=2, ref="blobs", blob_sigma=9.0),
}


@pytest.mark.parametrize("name", list(C2_CNN))
def test_mixed_precision_cnn_at_scale_every_member(cuda_ok, name):
    """Mixed-mode CNN at sizes where every CTA runs tens of row passes,
    checked against the FP64 oracle for every member, element by element:
    the increment X_next - X within 4u in relative L2 and 8u in max norm,
    u = 2^-9 (BF16 unit roundoff), per member and over the batch."""
    wl = C2_CNN[name]
    s = solver(wl, precision=oic.OIC_PREC_MIXED)
    rng = np.random.default_rng(17)
    X = (wl.X0()[None] + 0.3 * rng.standard_normal((wl.N, wl.n, wl.m))).astype(np.float32)
    U = (0.5 * rng.standard_normal((wl.N, wl.l, wl.m))).astype(np.float32)
    out = dev(np.zeros_like(X))
    s.oic_cnn_forward(dev(X), dev(U), out)
    s.oic_sync()
    got = out.cpu().numpy().astype(np.float64)
    want = oracle.cnn_step(onet(wl), X, U)
    inc = want - X
    u = 2.0 ** -9
    assert np.linalg.norm(got - want) <= 4 * u * np.linalg.norm(inc)
    assert np.abs(got - want).max() <= 8 * u * np.abs(inc).max()
    per_l2 = np.linalg.norm((got - want).reshape(wl.N, -1), axis=1) / np.linalg.norm(inc.reshape(wl.N, -1), axis=1)
    assert per_l2.max() <= 4 * u, (int(per_l2.argmax()), float(per_l2.max()))
    s.close()


def test_mixed_precision_fp64_gain_at_p144_matches_oracle(cuda_ok):
    """The mixed-mode analysis alone at p = n + l = 144 observed rows (the
    FP64 Cholesky's 18 panels wrap twice around its 8-CTA cluster) against
    the FP64 oracle's textbook analysis: relative L2 <= 1e-4 on the increment
    and on the ensemble mean (FP32 covariance products, FP64 gain)."""
    wl = W.large_128().with_(N=64)
    s = solver(wl, precision=oic.OIC_PREC_MIXED)
    rng = np.random.default_rng(23)
    R, p = 200, wl.p
    assert p == 144 and R <= s.max_rows
    E = (1.0 + 0.05 * rng.standard_normal((wl.N, R, wl.m))).astype(np.float32)
    obs = np.sort(rng.choice(R, size=p, replace=False))
    V = (0.02 * rng.standard_normal((wl.N, p, wl.m))).astype(np.float32)
    Ybar = (1.2 + 0.1 * rng.standard_normal((p, wl.m))).astype(np.float32)
    Ed = dev(E)
    s.oic_enks_update(Ed, obs, dev(V), dev(Ybar))
    assert s.oic_sync_status() == oic.OIC_OK
    got = Ed.cpu().numpy()
    want = oracle.enks_analysis(E, E[:, obs, :] + V, Ybar)
    assert rel(got - E, want - E) <= TOL
    assert rel(got.mean(0), want.mean(0)) <= TOL
    s.close()


C2_LOOP = W.large_128().with_(N=64, H=2, S=2)


@pytest.mark.slow
def test_mixed_precision_solve_128_matches_oracle(cuda_ok):
    """One mixed-mode horizon solve at 128 x 128, l = 16 (p = 144), CNN
    2-64-64-64-1, N = 64, H = 2, full history, against the FP64 oracle on the
    same noise: smoothed controls within 4u of BF16 (u = 2^-9) in relative L2,
    smoothed states within 1e-3."""
    wl = C2_LOOP
    s = solver(wl, precision=oic.OIC_PREC_MIXED, keep_full_history=True)
    Up = (0.01 * np.random.default_rng(29).standard_normal((wl.l, wl.m))).astype(np.float32)
    xr, ur, nz = wl.X_ref_window(1), wl.U_ref(), wl.noise(1)
    U_hat = np.zeros((wl.H + 1, wl.l, wl.m), np.float32)
    X_hat = np.zeros((wl.H + 1, wl.n, wl.m), np.float32)
    s.oic_solve_host(wl.X0(), Up, xr, ur, nz, U_hat, X_hat)
    xh = oracle.enks_solve(onet(wl), wl.N, wl.H, wl.X0(), Up, xr, ur, nz)
    assert rel(U_hat, xh[:, wl.n:wl.n + wl.l]) <= 4 * 2.0 ** -9
    assert rel(X_hat, xh[:, :wl.n]) <= 1e-3
    s.close()


@pytest.mark.slow
def test_mixed_precision_closed_loop_128_cost_within_half_percent(cuda_ok):
    """Two receding-horizon control steps of the mixed mode at 128 x 128
    (CNN 2-64-64-64-1, l = 16, N = 64, H = 2) against the FP64 oracle fed the
    same noise: cost J within 0.5%, applied controls within 4u, states within
    1e-3."""
    wl = C2_LOOP
    S = wl.S
    s = solver(wl, precision=oic.OIC_PREC_MIXED)
    xr_all = wl.X_ref_all(S)
    s.oic_reset_host(wl.X0(), wl.U_init())
    Ut = np.zeros((S, wl.l, wl.m), np.float32)
    Xt = np.zeros((S + 1, wl.n, wl.m), np.float32)
    Xt[0] = wl.X0()
    for k in range(S):
        s.oic_step_host(xr_all[k:k + wl.H + 1], wl.U_ref(), wl.noise(k), Ut[k], Xt[k + 1])
    Xo, Uo, _ = oracle.run(onet(wl), wl.N, wl.H, S, wl.X0(), wl.U_init(), xr_all, wl.U_ref(),
                           wl.noise_all(S))
    jg = oracle.closed_loop_cost(Xt, Ut, xr_all, wl.U_ref(), wl.U_init(), wl.sigma_vx, wl.sigma_vu,
                                 wl.sigma_w)
    jo = oracle.closed_loop_cost(Xo, Uo, xr_all, wl.U_ref(), wl.U_init(), wl.sigma_vx, wl.sigma_vu,
                                 wl.sigma_w)
    assert abs(jg - jo) <= 5e-3 * abs(jo)
    assert rel(Ut, Uo) <= 4 * 2.0 ** -9
    assert rel(Xt, Xo) <= 1e-3
    s.close()

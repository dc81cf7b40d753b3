"""The seeded input generator: deterministic, right shapes, right statistics."""
import numpy as np

from paper_2410_09663_b300 import workloads as W


def test_deterministic_and_shaped():
    wl = W.small_16()
    a, b = wl.noise(3), wl.noise(3)
    np.testing.assert_array_equal(a, b)
    assert a.dtype == np.float32 and a.size == wl.noise_floats()
    assert not np.array_equal(wl.noise(3), wl.noise(4))
    w1, b1 = wl.flat_weights()
    assert w1.size == sum(9 * ci * co for ci, co in zip(wl.channels[:-1], wl.channels[1:]))
    assert b1.size == sum(wl.channels[1:]) and np.all(b1 == 0)
    assert wl.B().shape == (wl.n, wl.l) and wl.X0().shape == (wl.n, wl.m)
    assert wl.X_ref_window(0).shape == (wl.H + 1, wl.n, wl.m)


def test_noise_statistics():
    wl = W.working_64().with_(N=64, H=3)
    z = wl.noise(0)
    assert abs(z.std() - 0.01) < 2e-4 and abs(z.mean()) < 1e-4


def test_reference_blobs_move_with_period_50():
    wl = W.working_64()
    r0, r25, r50 = wl.X_ref(0), wl.X_ref(25), wl.X_ref(50)
    np.testing.assert_allclose(r0, r50, atol=1e-6)
    # half a period swaps the two blobs: the field is symmetric under the swap
    np.testing.assert_allclose(r0, r25, atol=1e-5)
    assert 0.9 < r0.max() <= 1.05
    assert not np.allclose(r0, wl.X_ref(12))


def test_philox_known_answers():
    import json, os
    kat = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        ctr = np.array([[int(x, 16) for x in v["ctr"]]], np.uint32)
        key = [int(x, 16) for x in v["key"]]
        out = W.philox4x32_10(ctr, key)[0]
        assert [int(x) for x in out] == [int(x, 16) for x in v["out"]]


def test_philox_noise_layout_and_scale():
    wl = W.small_16().with_(sigma_vx=0.02)
    z = W.philox_noise(wl, solve=0)
    assert z.size == wl.noise_floats() and z.dtype == np.float32
    e1 = wl.N * wl.l * wl.m + wl.H * wl.N * wl.l * wl.m
    e2 = e1 + wl.H * wl.N * wl.n * wl.m
    assert abs(z[:e1].std() - 0.01) < 1e-3 and abs(z[e1:e2].std() - 0.02) < 1e-3
    assert not np.array_equal(W.philox_noise(wl, 0), W.philox_noise(wl, 1))

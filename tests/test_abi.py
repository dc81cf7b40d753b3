"""The C ABI library loads, exports every symbol include/oic.h declares, and
validates configurations on the host (no device work is started here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2410_09663_b300 as oic
from paper_2410_09663_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(oic_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = oic.load()
    names = _declared_symbols()
    assert len(names) >= 15
    for name in sorted(names):
        assert hasattr(lib, name), name


def test_status_strings_and_version():
    lib = oic.load()
    assert b"sm_103a" in lib.oic_version()
    for s in range(7):
        assert oic.status_string(s)


def _create(cfg, wl):
    lib = oic.load()
    w, b = wl.flat_weights()
    B = wl.B()
    h = ctypes.c_void_p()
    st = lib.oic_create(ctypes.byref(cfg), w.ctypes.data, b.ctypes.data, B.ctypes.data, ctypes.byref(h))
    return st, h


def test_create_accepts_workloads_and_sizes_workspace():
    lib = oic.load()
    for name in ("small_16", "working_64", "large_128"):
        wl = W.WORKLOADS[name]()
        cfg = oic.config_from_workload(wl)
        assert lib.oic_noise_floats(ctypes.byref(cfg)) == wl.noise_floats()
        st, h = _create(cfg, wl)
        assert st == oic.OIC_OK
        ws = lib.oic_workspace_bytes(h)
        # at least the ensemble, the activations and the noise staging
        ens = wl.N * (2 * wl.n + (wl.H + 1) * wl.l) * wl.m * 4
        act = 2 * wl.N * max(wl.channels[1:-1]) * wl.n * wl.m * 4
        assert ws >= ens + act + wl.noise_floats() * 4
        assert lib.oic_max_rows(h) == wl.n + (wl.H + 1) * wl.l
        lib.oic_destroy(h)


@pytest.mark.parametrize("field,value", [("n", 0), ("m", 6), ("l", 0), ("N", 1), ("H", 0),
                                          ("n_layers", 0), ("precision", 7), ("noise_mode", 3)])
def test_create_rejects_bad_config(field, value):
    wl = W.small_16()
    cfg = oic.config_from_workload(wl)
    setattr(cfg, field, value)
    st, h = _create(cfg, wl)
    assert st == oic.OIC_EINVAL and not h.value


def test_create_rejects_bad_channels_and_null_pointers():
    lib = oic.load()
    wl = W.small_16()
    cfg = oic.config_from_workload(wl)
    cfg.channels[0] = 3
    assert _create(cfg, wl)[0] == oic.OIC_EINVAL
    cfg = oic.config_from_workload(wl)
    h = ctypes.c_void_p()
    assert lib.oic_create(ctypes.byref(cfg), None, None, None, ctypes.byref(h)) == oic.OIC_EINVAL


def test_unbound_handle_reports_state_error():
    lib = oic.load()
    wl = W.small_16()
    st, h = _create(oic.config_from_workload(wl), wl)
    assert st == oic.OIC_OK
    x = np.zeros(16, np.float32)
    assert lib.oic_solve(h, x.ctypes.data, x.ctypes.data, x.ctypes.data, x.ctypes.data,
                         x.ctypes.data, x.ctypes.data, None) == oic.OIC_ESTATE
    assert lib.oic_step(h, x.ctypes.data, x.ctypes.data, x.ctypes.data, None, None) == oic.OIC_ESTATE
    assert lib.oic_bind(h, None, 0, None) == oic.OIC_EINVAL
    lib.oic_destroy(h)


def _constraints(c_spec, alpha=None):
    arrs = [np.ascontiguousarray(a, np.float32).ravel() for a in (c_spec.Gx, c_spec.Gu, c_spec.h)]
    cs = oic.oic_constraints()
    cs.c = int(arrs[2].size)
    cs.Gx, cs.Gu, cs.h = (a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) for a in arrs)
    cs.alpha = c_spec.alpha if alpha is None else alpha
    cs.beta, cs.sigma_z = c_spec.beta, c_spec.sigma_z
    return cs, arrs


def _create_constrained(wl, cs):
    lib = oic.load()
    cfg = oic.config_from_workload(wl)
    w, b = wl.flat_weights()
    B = wl.B()
    h = ctypes.c_void_p()
    s = lib.oic_create_constrained(ctypes.byref(cfg), w.ctypes.data, b.ctypes.data, B.ctypes.data,
                                   None if cs is None else ctypes.byref(cs), ctypes.byref(h))
    return s, h


def test_constrained_create_sizes_noise_and_workspace():
    lib = oic.load()
    wl = W.small_16()
    s0, h0 = _create_constrained(wl, None)
    wc = wl.with_(cons=W.u_box(wl.n, wl.l, 0.1))
    cs, keep = _constraints(wc.cons)
    s1, h1 = _create_constrained(wl, cs)
    try:
        assert s0 == s1 == oic.OIC_OK
        assert lib.oic_handle_noise_floats(h0) == wl.noise_floats()
        assert lib.oic_handle_noise_floats(h1) == wc.noise_floats() == wl.noise_floats() + wl.H * wl.N * 2 * wl.l * wl.m
        assert lib.oic_workspace_bytes(h1) > lib.oic_workspace_bytes(h0)
    finally:
        lib.oic_destroy(h0)
        lib.oic_destroy(h1)


def test_constrained_create_rejects_bad_constraints():
    wl = W.small_16()
    spec = W.u_box(wl.n, wl.l, 0.1)
    for alpha in (0.0, -1.0):
        cs, keep = _constraints(spec, alpha=alpha)
        assert _create_constrained(wl, cs)[0] == oic.OIC_EINVAL
    cs, keep = _constraints(spec)
    cs.beta = 0.0
    assert _create_constrained(wl, cs)[0] == oic.OIC_EINVAL
    cs, keep = _constraints(spec)
    cs.Gu = ctypes.POINTER(ctypes.c_float)()
    assert _create_constrained(wl, cs)[0] == oic.OIC_EINVAL
    # n + l + c <= 144
    big = W.Workload("b", n=128, m=16, l=8, channels=[2, 4, 1], N=8, H=2, S=1)
    cs, keep = _constraints(W.u_box(big.n, big.l, 0.1))          # c = 16
    assert _create_constrained(big, cs)[0] == oic.OIC_EINVAL
    edge = W.Constraints(np.zeros((8, big.n), np.float32), np.eye(8, dtype=np.float32),
                         np.full(8, 0.1, np.float32))                 # c = 8: 128 + 8 + 8 = 144
    cs, keep = _constraints(edge)
    s, h = _create_constrained(big, cs)
    assert s == oic.OIC_OK
    oic.load().oic_destroy(h)

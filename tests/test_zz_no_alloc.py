"""oic_enks_update_static: the ensemble Kalman analysis for callers that
cannot allocate device memory (real-time loops that must never reach the
allocator after start-up, plug-ins whose host application owns the GPU
memory pool).  It keeps all of its scratch in a fixed device array inside the
library, so its results must equal those of the workspace-based
oic_enks_update -- and the FP64 oracle's analysis -- call after call, even
though every call reuses (and leaves behind) the same scratch.

This file is collected last so a failure here never hides the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2410_09663_b300 as oic
from paper_2410_09663_b300 import workloads as W

TOL = 1e-4


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _call_static(lib, E, obs, V, Ybar, stream):
    rows = np.ascontiguousarray(obs, np.int32)
    N, R, m = E.shape
    return lib.oic_enks_update_static(N, R, m, len(rows), rows.ctypes.data, ctypes.c_void_p(E.data_ptr()),
                                      ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(Ybar.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream))


def test_static_sizes_rejected_without_device_work():
    lib = oic.load()
    x = np.zeros(4, np.float32)
    rows = np.zeros(8, np.int32)
    # far beyond the fixed scratch: refused on the host before any launch
    st = lib.oic_enks_update_static(1 << 16, 100, 128, 8, rows.ctypes.data, x.ctypes.data, x.ctypes.data,
                                    x.ctypes.data, None)
    assert st in (oic.OIC_ENOMEM, oic.OIC_EINVAL)
    st = lib.oic_enks_update_static(1 << 16, 100, 128, 8, rows.ctypes.data, None, None, None, None)
    assert st == oic.OIC_EINVAL


@pytest.mark.gpu
def test_static_scratch_update_matches_workspace_update_twice(cuda_ok):
    import torch
    lib = oic.load()
    wl = W.Workload("noalloc_32x48", n=32, m=48, l=4, channels=[2, 16, 16, 1], N=64, H=4, S=1)
    w, b = wl.flat_weights()
    s = oic.Solver(oic.config_from_workload(wl), w, b, wl.B())
    stream = torch.cuda.current_stream()
    R, p = 45, wl.p
    for call in range(2):                       # the second call runs on the first call's leftovers
        rng = np.random.default_rng(100 + call)
        E = (1.0 + 0.05 * rng.standard_normal((wl.N, R, wl.m))).astype(np.float32)
        obs = np.sort(rng.choice(R, size=p, replace=False))
        V = (0.02 * rng.standard_normal((wl.N, p, wl.m))).astype(np.float32)
        Ybar = (1.2 + 0.1 * rng.standard_normal((p, wl.m))).astype(np.float32)
        Vd, Yd = torch.from_numpy(V).cuda(), torch.from_numpy(Ybar).cuda()
        E_ref = torch.from_numpy(E).cuda()
        s.oic_enks_update(E_ref, obs, Vd, Yd)
        s.oic_sync()
        E_st = torch.from_numpy(E).cuda()
        assert _call_static(lib, E_st, obs, Vd, Yd, stream) == oic.OIC_OK
        ref, got = E_ref.cpu().numpy(), E_st.cpu().numpy()
        assert _rel(got - E, ref - E) <= TOL
        assert _rel(got.mean(0), ref.mean(0)) <= TOL
        want = oracle.enks_analysis(E, E[:, obs, :] + V, Ybar)
        assert _rel(got - E, want - E) <= TOL
        assert _rel(got.mean(0), want.mean(0)) <= TOL


@pytest.mark.gpu
def test_static_refuses_host_pointers(cuda_ok):
    """E, V and Ybar must be memory of the current device: pageable host
    arrays are refused on the host, before anything is launched."""
    import torch
    lib = oic.load()
    N, R, m, p = 4, 8, 16, 4
    rows = np.arange(p, dtype=np.int32)
    E = np.ones((N, R, m), np.float32)
    V = np.zeros((N, p, m), np.float32)
    Y = np.zeros((p, m), np.float32)
    st = lib.oic_enks_update_static(N, R, m, p, rows.ctypes.data, E.ctypes.data, V.ctypes.data, Y.ctypes.data,
                                    None)
    assert st == oic.OIC_EINVAL
    Ed = torch.from_numpy(E).cuda()
    st = lib.oic_enks_update_static(N, R, m, p, rows.ctypes.data, ctypes.c_void_p(Ed.data_ptr()), V.ctypes.data,
                                    Y.ctypes.data, None)
    assert st == oic.OIC_EINVAL
    np.testing.assert_array_equal(Ed.cpu().numpy(), E)

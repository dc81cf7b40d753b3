"""paper_2410_09663_b300 -- Kalman-MPC (arXiv 2410.09663) on one B300 GPU.

Thin ctypes binding over ``liboic.so`` (C ABI in ``include/oic.h``).  The
functions below carry the C names and only marshal arguments: every step of
the method runs in the library's CUDA kernels.  PyTorch is used for device
memory and streams (``Solver`` allocates the workspace with torch and binds
it).  There is no CPU fallback: if the library cannot be loaded every call
raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

__all__ = ["OIC_OK", "OICError", "oic_config", "load", "Solver", "Batch", "config_from_workload"]

MAX_LAYERS = 8
OIC_OK, OIC_EINVAL, OIC_ENOMEM, OIC_ECUDA, OIC_ENOTSPD, OIC_ETIMEOUT, OIC_ESTATE = range(7)
OIC_PREC_FP32, OIC_PREC_MIXED = 0, 1
OIC_NOISE_HOST, OIC_NOISE_PHILOX = 0, 1
STAGES = ["noise", "init", "cnn_input", "conv_first", "conv_hidden", "conv_out", "u_advance",
          "means", "cov", "cov_reduce", "gain", "update", "block_means", "cnn_fused", "cnn_bf16",
          "constraint", "cov_out"]


class OICError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = int(status)
        super().__init__(f"{what}: {status_string(status)} (status {status})")


class oic_config(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("m", ctypes.c_int), ("l", ctypes.c_int), ("N", ctypes.c_int),
        ("H", ctypes.c_int), ("n_layers", ctypes.c_int),
        ("channels", ctypes.c_int * (MAX_LAYERS + 1)),
        ("residual_scale", ctypes.c_float),
        ("sigma_w", ctypes.c_double), ("sigma_vx", ctypes.c_double), ("sigma_vu", ctypes.c_double),
        ("precision", ctypes.c_int), ("keep_full_history", ctypes.c_int), ("noise_mode", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
    ]


class oic_constraints(ctypes.Structure):
    _fields_ = [
        ("c", ctypes.c_int),
        ("Gx", ctypes.POINTER(ctypes.c_float)), ("Gu", ctypes.POINTER(ctypes.c_float)),
        ("h", ctypes.POINTER(ctypes.c_float)),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("sigma_z", ctypes.c_double),
    ]


class oic_plan(ctypes.Structure):
    _fields_ = [("stats_splits", ctypes.c_int), ("update_ctas", ctypes.c_int), ("cnn_ctas", ctypes.c_int)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


OIC_TUNE_FORCE = 1

_lib = None
_VP = ctypes.c_void_p
_FP = ctypes.POINTER(ctypes.c_float)

_SIGS = {
    "oic_noise_floats": (ctypes.c_size_t, [ctypes.POINTER(oic_config)]),
    "oic_create": (ctypes.c_int, [ctypes.POINTER(oic_config), _VP, _VP, _VP, ctypes.POINTER(_VP)]),
    "oic_create_constrained": (ctypes.c_int, [ctypes.POINTER(oic_config), _VP, _VP, _VP,
                                              ctypes.POINTER(oic_constraints), ctypes.POINTER(_VP)]),
    "oic_handle_noise_floats": (ctypes.c_size_t, [_VP]),
    "oic_solve_cov": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_double, _VP, _VP, _VP,
                                     ctypes.c_size_t]),
    "oic_cov_scratch_bytes": (ctypes.c_size_t, [_VP]),
    "oic_cov_rows": (ctypes.c_int, [_VP, ctypes.c_int]),
    "oic_workspace_bytes": (ctypes.c_size_t, [_VP]),
    "oic_max_rows": (ctypes.c_int, [_VP]),
    "oic_bind": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t, _VP]),
    "oic_reset": (ctypes.c_int, [_VP, _VP, _VP]),
    "oic_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "oic_step": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "oic_reset_host": (ctypes.c_int, [_VP, _VP, _VP]),
    "oic_solve_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "oic_step_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "oic_cnn_forward": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    "oic_enks_update": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "oic_sync": (ctypes.c_int, [_VP]),
    "oic_last_ms": (ctypes.c_float, [_VP]),
    "oic_profile_begin": (ctypes.c_int, [_VP, ctypes.c_uint, ctypes.c_int]),
    "oic_profile_end": (ctypes.c_int, [_VP, _FP, ctypes.POINTER(ctypes.c_int)]),
    "oic_profile_sample": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "oic_launch_count": (ctypes.c_ulonglong, []),
    "oic_get_plan": (ctypes.c_int, [_VP, ctypes.POINTER(oic_plan), ctypes.POINTER(oic_plan)]),
    "oic_set_plan": (ctypes.c_int, [_VP, ctypes.POINTER(oic_plan)]),
    "oic_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(oic_plan),
                                    ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "oic_selftest": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "oic_enks_update_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP,
                                              _VP, _VP, _VP]),
    "oic_control_expand": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP]),
    "oic_control_reduce": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP]),
    "oic_state_bytes": (ctypes.c_size_t, [_VP]),
    "oic_save_state": (ctypes.c_int, [_VP, _VP]),
    "oic_load_state": (ctypes.c_int, [_VP, _VP]),
    "oic_io_slots": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "oic_batch_create": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP]),
    "oic_batch_step": (ctypes.c_int, [_VP]),
    "oic_batch_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_float)]),
    "oic_batch_sync": (ctypes.c_int, [_VP]),
    "oic_batch_destroy": (None, [_VP]),
    "oic_destroy": (None, [_VP]),
    "oic_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "oic_version": (ctypes.c_char_p, []),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liboic.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise OSError(f"liboic.so not found at {path}; run python -m paper_2410_09663_b300.build")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        _lib = lib
    return _lib


def oic_launch_count() -> int:
    return int(load().oic_launch_count())


def status_string(s) -> str:
    return load().oic_status_string(int(s)).decode()


def _check(s, what):
    if s != OIC_OK:
        raise OICError(s, what)


class Batch:
    """oic_batch: one control step of several independent solvers as one
    CUDA graph (each solver's step graph a branch).  Inputs go into each
    solver's oic_io_slots() views before step(); outputs are read there."""

    def __init__(self, solvers, stream=None):
        import torch
        self._lib = load()
        self.solvers = list(solvers)
        dev = self.solvers[0].workspace.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        arr = (ctypes.c_void_p * len(self.solvers))(*[sv.h for sv in self.solvers])
        b = ctypes.c_void_p()
        _check(self._lib.oic_batch_create(arr, len(self.solvers), ctypes.c_void_p(self.stream.cuda_stream),
                                          ctypes.byref(b)), "oic_batch_create")
        self.b = b

    def step(self):
        _check(self._lib.oic_batch_step(self.b), "oic_batch_step")

    def autotune(self, reps=3):
        """One plan for all problems chosen by timing batch steps; returns
        (ms per batch step with the rules, with the chosen plans)."""
        a, b = ctypes.c_float(), ctypes.c_float()
        _check(self._lib.oic_batch_autotune(self.b, int(reps), ctypes.byref(a), ctypes.byref(b)),
               "oic_batch_autotune")
        return float(a.value), float(b.value)

    def sync(self):
        _check(self._lib.oic_batch_sync(self.b), "oic_batch_sync")

    def close(self):
        if getattr(self, "b", None):
            self._lib.oic_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_of(t, stream):
    import torch
    st = stream if stream is not None else torch.cuda.current_stream(t.device)
    return ctypes.c_void_p(st.cuda_stream)


def oic_control_expand(u, T, U, stream=None):
    """U = u T for a control u [l, mu] with fewer columns than the state
    (T [mu, m]); device tensors, float32, asynchronous on `stream`."""
    l, mu = u.shape
    _check(load().oic_control_expand(_ptr(u), l, mu, _ptr(T), T.shape[1], _ptr(U), _stream_of(u, stream)),
           "oic_control_expand")


def oic_control_reduce(U, T, u, stream=None):
    """u = U T^T (T T^T)^{-1} (U [l, m], T [mu, m]); waits for the stream."""
    l, m = U.shape
    _check(load().oic_control_reduce(_ptr(U), l, m, _ptr(T), T.shape[0], _ptr(u), _stream_of(U, stream)),
           "oic_control_reduce")


def config_from_workload(wl, precision=OIC_PREC_FP32, keep_full_history=False,
                         noise_mode=OIC_NOISE_HOST, seed=None) -> oic_config:
    c = oic_config()
    c.n, c.m, c.l, c.N, c.H = wl.n, wl.m, wl.l, wl.N, wl.H
    c.n_layers = len(wl.channels) - 1
    for k, ch in enumerate(wl.channels):
        c.channels[k] = ch
    c.residual_scale = wl.residual_scale
    c.sigma_w, c.sigma_vx, c.sigma_vu = wl.sigma_w, wl.sigma_vx, wl.sigma_vu
    c.precision = precision
    c.keep_full_history = int(bool(keep_full_history))
    c.noise_mode = noise_mode
    c.seed = wl.seed if seed is None else seed
    return c


def _ptr(t):
    """Device or host address of a torch tensor (None -> NULL)."""
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Solver:
    """Owns an oic_handle plus a torch-allocated device workspace.

    Methods mirror the C entry points; tensors are passed by address.
    """

    def __init__(self, cfg: oic_config, conv_w, conv_b, B, device="cuda", stream=None, constraints=None):
        """constraints: None, or an object with Gx (c x n), Gu (c x l), h (c),
        alpha, beta, sigma_z (workloads.Constraints) -> oic_create_constrained."""
        import numpy as np
        import torch
        lib = load()
        self._lib = lib
        self.cfg = cfg
        w = np.ascontiguousarray(conv_w, dtype=np.float32)
        b = np.ascontiguousarray(conv_b, dtype=np.float32)
        Bm = np.ascontiguousarray(B, dtype=np.float32)
        h = _VP()
        cs = None
        if constraints is not None:
            self._cons_arrays = [np.ascontiguousarray(a, dtype=np.float32).ravel()
                                 for a in (constraints.Gx, constraints.Gu, constraints.h)]
            cs = oic_constraints()
            cs.c = int(self._cons_arrays[2].size)
            cs.Gx, cs.Gu, cs.h = (a.ctypes.data_as(_FP) for a in self._cons_arrays)
            cs.alpha, cs.beta, cs.sigma_z = float(constraints.alpha), float(constraints.beta), \
                float(constraints.sigma_z)
        _check(lib.oic_create_constrained(ctypes.byref(cfg), w.ctypes.data, b.ctypes.data, Bm.ctypes.data,
                                          None if cs is None else ctypes.byref(cs), ctypes.byref(h)),
               "oic_create")
        self.h = h
        self.ws_bytes = lib.oic_workspace_bytes(h)
        self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        _check(lib.oic_bind(h, ctypes.c_void_p(self._ws_ptr), self.ws_bytes,
                            ctypes.c_void_p(self.stream.cuda_stream)), "oic_bind")

    # -- sizes
    @property
    def noise_floats(self):
        return self._lib.oic_handle_noise_floats(self.h)

    @property
    def max_rows(self):
        return self._lib.oic_max_rows(self.h)

    # -- device-pointer entry points (asynchronous on self.stream)
    def oic_reset(self, X0, U_prev):
        _check(self._lib.oic_reset(self.h, _ptr(X0), _ptr(U_prev)), "oic_reset")

    def oic_solve(self, X_k, U_prev, X_ref, U_ref, noise, U_hat, X_hat=None):
        _check(self._lib.oic_solve(self.h, _ptr(X_k), _ptr(U_prev), _ptr(X_ref), _ptr(U_ref),
                                   _ptr(noise), _ptr(U_hat), _ptr(X_hat)), "oic_solve")

    def oic_solve_cov(self, X_k, U_prev, X_ref, U_ref, noise, U_hat, X_hat=None, lam=1.0, Sigma_pred=None,
                      Sigma_post=None):
        """oic_solve plus the optional covariance outputs (float64 device
        tensors of H * R * R, R = oic_cov_rows(H)); scratch is allocated here."""
        import torch
        nb = int(self._lib.oic_cov_scratch_bytes(self.h))
        scratch = torch.empty(nb + 256, dtype=torch.uint8, device=self.workspace.device)
        sp = (scratch.data_ptr() + 255) // 256 * 256
        _check(self._lib.oic_solve_cov(self.h, _ptr(X_k), _ptr(U_prev), _ptr(X_ref), _ptr(U_ref), _ptr(noise),
                                       _ptr(U_hat), _ptr(X_hat), float(lam), _ptr(Sigma_pred), _ptr(Sigma_post),
                                       ctypes.c_void_p(sp), nb), "oic_solve_cov")
        self._cov_scratch = scratch                  # alive until the stream has used it

    def oic_cov_rows(self, s):
        return int(self._lib.oic_cov_rows(self.h, int(s)))

    def oic_step(self, X_ref, U_ref, noise, U_applied=None, X_next=None):
        _check(self._lib.oic_step(self.h, _ptr(X_ref), _ptr(U_ref), _ptr(noise), _ptr(U_applied),
                                  _ptr(X_next)), "oic_step")

    def oic_cnn_forward(self, X, U, X_next):
        batch = X.shape[0]
        _check(self._lib.oic_cnn_forward(self.h, batch, _ptr(X), _ptr(U), _ptr(X_next)),
               "oic_cnn_forward")

    def oic_enks_update(self, E, obs_rows, V, Ybar):
        import numpy as np
        rows = np.ascontiguousarray(obs_rows, dtype=np.int32)
        _check(self._lib.oic_enks_update(self.h, int(E.shape[1]), rows.ctypes.data, _ptr(E), _ptr(V),
                                         _ptr(Ybar)), "oic_enks_update")

    # -- host-pointer entry points (synchronous); arguments are numpy arrays
    def oic_reset_host(self, X0, U_prev):
        import numpy as np
        X0 = np.ascontiguousarray(X0, np.float32)
        U_prev = np.ascontiguousarray(U_prev, np.float32)
        _check(self._lib.oic_reset_host(self.h, X0.ctypes.data, U_prev.ctypes.data), "oic_reset_host")

    def oic_solve_host(self, X_k, U_prev, X_ref, U_ref, noise, U_hat, X_hat=None):
        import numpy as np
        a = [np.ascontiguousarray(x, np.float32) for x in (X_k, U_prev, X_ref, U_ref)]
        nz = None if noise is None else np.ascontiguousarray(noise, np.float32)
        _check(self._lib.oic_solve_host(self.h, *[x.ctypes.data for x in a],
                                        None if nz is None else nz.ctypes.data, U_hat.ctypes.data,
                                        None if X_hat is None else X_hat.ctypes.data),
               "oic_solve_host")

    def oic_step_host(self, X_ref, U_ref, noise, U_applied=None, X_next=None):
        import numpy as np
        xr = np.ascontiguousarray(X_ref, np.float32)
        ur = np.ascontiguousarray(U_ref, np.float32)
        nz = None if noise is None else np.ascontiguousarray(noise, np.float32)
        _check(self._lib.oic_step_host(self.h, xr.ctypes.data, ur.ctypes.data,
                                       None if nz is None else nz.ctypes.data,
                                       None if U_applied is None else U_applied.ctypes.data,
                                       None if X_next is None else X_next.ctypes.data),
               "oic_step_host")

    def oic_step_host_ptr(self, X_ref_ptr, U_ref_ptr, noise_ptr, U_applied_ptr, X_next_ptr):
        """oic_step_host with raw host addresses (e.g. pinned torch tensors)."""
        _check(self._lib.oic_step_host(self.h, X_ref_ptr, U_ref_ptr, noise_ptr, U_applied_ptr,
                                       X_next_ptr), "oic_step_host")

    def oic_selftest(self):
        """Returns (status, [mismatches, row, col, got, want])."""
        res = (ctypes.c_int * 5)()
        st = self._lib.oic_selftest(self.h, res)
        return int(st), list(res)

    def oic_get_plan(self):
        """(plan in use with rules resolved, limits) as dicts."""
        pl, lim = oic_plan(), oic_plan()
        _check(self._lib.oic_get_plan(self.h, ctypes.byref(pl), ctypes.byref(lim)), "oic_get_plan")
        return pl.as_dict(), lim.as_dict()

    def oic_set_plan(self, stats_splits=0, update_ctas=0, cnn_ctas=0):
        pl = oic_plan(stats_splits, update_ctas, cnn_ctas)
        _check(self._lib.oic_set_plan(self.h, ctypes.byref(pl)), "oic_set_plan")

    def oic_autotune(self, reps=3, force=False):
        """Returns (chosen plan dict, ms per step with the rule plan, with the
        chosen plan); both times are -1 when the plan came from the cache."""
        pl = oic_plan()
        a, b = ctypes.c_float(), ctypes.c_float()
        _check(self._lib.oic_autotune(self.h, int(reps), OIC_TUNE_FORCE if force else 0, ctypes.byref(pl),
                                      ctypes.byref(a), ctypes.byref(b)), "oic_autotune")
        return pl.as_dict(), float(a.value), float(b.value)

    def oic_sync(self):
        _check(self._lib.oic_sync(self.h), "oic_sync")

    def oic_sync_status(self) -> int:
        return int(self._lib.oic_sync(self.h))

    def oic_last_ms(self) -> float:
        return float(self._lib.oic_last_ms(self.h))

    def oic_profile_begin(self, stages=None, max_launches=100000):
        mask = 0
        for st in (STAGES if stages is None else stages):
            mask |= 1 << STAGES.index(st)
        _check(self._lib.oic_profile_begin(self.h, mask, int(max_launches)), "oic_profile_begin")

    def oic_profile_sample(self, every, phase=0):
        """Bracket only launch i of a profiled stage in a solve with
        i % every == phase (oic_profile_sample)."""
        _check(self._lib.oic_profile_sample(self.h, int(every), int(phase)), "oic_profile_sample")

    def oic_profile_end(self):
        """Returns {stage: (total_ms, launches)} for the profiled stages."""
        n = len(STAGES)
        ms = (ctypes.c_float * n)()
        cnt = (ctypes.c_int * n)()
        _check(self._lib.oic_profile_end(self.h, ms, cnt), "oic_profile_end")
        return {STAGES[i]: (float(ms[i]), int(cnt[i])) for i in range(n) if cnt[i] > 0}

    def oic_save_state(self):
        """The problem's state (plant X, last control, solve index) as bytes."""
        buf = ctypes.create_string_buffer(int(self._lib.oic_state_bytes(self.h)))
        _check(self._lib.oic_save_state(self.h, buf), "oic_save_state")
        return buf.raw

    def oic_load_state(self, state: bytes):
        buf = ctypes.create_string_buffer(state, len(state))
        _check(self._lib.oic_load_state(self.h, buf), "oic_load_state")
        self.stream.synchronize()                       # the buffer is local

    def oic_io_slots(self):
        """Torch views of the per-step slots in this solver's workspace:
        (X_ref [H+1, n, m], U_ref [l, m], U_applied [l, m], X_next [n, m])."""
        import torch
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        _check(self._lib.oic_io_slots(self.h, *[ctypes.byref(q) for q in ptrs]), "oic_io_slots")
        c = self.cfg
        shapes = [(c.H + 1, c.n, c.m), (c.l, c.m), (c.l, c.m), (c.n, c.m)]
        base = self.workspace.data_ptr()
        out = []
        for q, shp in zip(ptrs, shapes):
            off = q.value - base
            n = 4
            for d in shp:
                n *= d
            out.append(self.workspace[off:off + n].view(torch.float32).view(*shp))
        return tuple(out)

    def close(self):
        if getattr(self, "h", None):
            self._lib.oic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Serving loop for receding-horizon control requests: continuous batching of
independent problems on one GPU, above the C ABI.

A request asks for the next control step of one problem (Algorithm 1 of
arXiv 2410.09663 applied once: solve, apply U_k, advance the plant).  The
server keeps every admitted problem device-resident between its steps, on
its own CUDA stream, so requests of different problems that arrive while
others are on the GPU run side by side; the steps of one problem run in
arrival order, one at a time.

Admission is by HBM footprint: a problem's workspace (``oic_workspace_bytes``)
is allocated when it is admitted and counted against the budget.  When a
problem with waiting requests does not fit, idle problems (nothing queued or
running) are evicted, least recently used first: their state (plant X, last
control, Philox solve index; ``oic_save_state``) goes to the host and comes
back into a fresh handle on re-admission, so every step is bit-identical to
the same problem served alone and uninterrupted.
"""
from __future__ import annotations

import collections
import ctypes
import time

import numpy as np

from . import OIC_NOISE_PHILOX, Solver, config_from_workload, load


def workspace_bytes(cfg) -> int:
    """Device bytes a handle of this configuration needs (host-side query)."""
    lib = load()
    h = ctypes.c_void_p()
    # the weights only matter for the packed tiles' contents, not their size
    Lw = sum(cfg.channels[k + 1] * cfg.channels[k] * 9 for k in range(cfg.n_layers))
    Lb = sum(cfg.channels[k + 1] for k in range(cfg.n_layers))
    w = np.zeros(Lw, np.float32)
    b = np.zeros(Lb, np.float32)
    B = np.zeros(cfg.n * cfg.l, np.float32)
    s = lib.oic_create(ctypes.byref(cfg), w.ctypes.data, b.ctypes.data, B.ctypes.data, ctypes.byref(h))
    if s != 0:
        raise RuntimeError(f"oic_create: status {s}")
    try:
        return int(lib.oic_workspace_bytes(h))
    finally:
        lib.oic_destroy(h)


class Problem:
    """One control problem: its workload, its solver while resident, its saved
    state while evicted, its queue of waiting requests."""

    def __init__(self, pid, wl, precision, steps_max):
        self.pid, self.wl, self.precision = pid, wl, precision
        self.cfg = config_from_workload(wl, precision=precision, noise_mode=OIC_NOISE_PHILOX)
        self.steps_max = steps_max
        self.ref_host = wl.X_ref_all(steps_max)         # references of every step it may serve
        # device footprint: the workspace, the references, the step's outputs
        self.bytes = workspace_bytes(self.cfg) + self.ref_host.nbytes + 4 * (wl.n + 2 * wl.l) * wl.m
        self.solver = None
        self.stream = None
        self.refs = None
        self.state = None                   # saved state while evicted
        self.queue = collections.deque()    # request indices
        self.running = None                 # (request index, done event)
        self.k = 0                          # next control step
        self.last_used = 0.0
        self.evictions = 0
        self.u_out = self.x_out = None


class Server:
    def __init__(self, device, budget_bytes, precision, max_running=64, keep_outputs=False):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.budget = int(budget_bytes)
        self.precision = precision
        self.max_running = max_running
        self.keep_outputs = keep_outputs
        self.problems = {}
        self.used = 0

    def add(self, pid, wl, steps_max):
        self.problems[pid] = Problem(pid, wl, self.precision, steps_max)

    # ------------------------------------------------------------ residency
    def _admit(self, p, now):
        torch = self.torch
        if p.bytes > self.budget:
            raise RuntimeError(f"problem {p.pid} needs {p.bytes} bytes, more than the budget")
        if self.used + p.bytes > self.budget:
            idle = sorted((q for q in self.problems.values()
                           if q.solver is not None and q.running is None and not q.queue),
                          key=lambda q: q.last_used)
            for q in idle:
                if self.used + p.bytes <= self.budget:
                    break
                self._evict(q)
            if self.used + p.bytes > self.budget:
                return False                # wait until running problems finish
        p.stream = torch.cuda.Stream(device=self.device)
        w, b = p.wl.flat_weights()
        with torch.cuda.stream(p.stream):
            p.solver = Solver(p.cfg, w, b, p.wl.B(), device=self.device, stream=p.stream)
            if p.state is None:
                p.solver.oic_reset(torch.from_numpy(p.wl.X0()).to(self.device),
                                   torch.from_numpy(p.wl.U_init()).to(self.device))
            else:
                p.solver.oic_load_state(p.state)
            p.refs = torch.from_numpy(p.ref_host).to(self.device)
            p.uref = torch.zeros(p.wl.l, p.wl.m, device=self.device)
            p.u_out = torch.zeros(p.wl.l, p.wl.m, device=self.device)
            p.x_out = torch.zeros(p.wl.n, p.wl.m, device=self.device)
        self.used += p.bytes
        p.last_used = now
        return True

    def _evict(self, p):
        p.state = p.solver.oic_save_state()
        p.solver.close()
        p.solver = None
        p.refs = p.uref = p.u_out = p.x_out = None
        self.used -= p.bytes
        p.evictions += 1

    # ---------------------------------------------------------------- loop
    def run(self, arrivals):
        """Serve `arrivals` = [(arrival time in s, problem id)] in real time.
        Returns one record per request: (pid, step, arrival, start, done) in
        seconds from the start, plus U_applied if keep_outputs.  Afterwards
        `device_intervals[i]` holds (start, end) in ms of request i's work on
        the GPU (CUDA events on the problem's stream, relative to an event
        recorded when the run began), from which overlap on the device is
        measured."""
        torch = self.torch
        order = sorted(range(len(arrivals)), key=lambda i: arrivals[i][0])
        rec = [None] * len(arrivals)
        outs = [None] * len(arrivals)
        evs = [None] * len(arrivals)
        running = []
        nxt, left = 0, len(arrivals)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev0.record(torch.cuda.current_stream(self.device))
        t0 = time.perf_counter()
        while left:
            now = time.perf_counter() - t0
            while nxt < len(order) and arrivals[order[nxt]][0] <= now:
                i = order[nxt]
                self.problems[arrivals[i][1]].queue.append(i)
                nxt += 1
            # completions
            still = []
            for p in running:
                i, ev, t_start = p.running
                if ev.query():
                    t_done = time.perf_counter() - t0
                    rec[i] = (p.pid, p.k, arrivals[i][0], t_start, t_done)
                    if self.keep_outputs:
                        outs[i] = p.u_out.cpu().numpy()
                    p.running = None
                    p.k += 1
                    p.last_used = t_done
                    left -= 1
                else:
                    still.append(p)
            running = still
            # launches: the problems whose oldest request arrived first
            ready = sorted((p for p in self.problems.values() if p.queue and p.running is None),
                           key=lambda p: arrivals[p.queue[0]][0])
            for p in ready:
                if len(running) >= self.max_running:
                    break
                if p.solver is None and not self._admit(p, now):
                    continue
                i = p.queue.popleft()
                k = p.k
                with torch.cuda.stream(p.stream):
                    ev_start = torch.cuda.Event(enable_timing=True)
                    ev_start.record(p.stream)
                    p.solver.oic_step(p.refs[k:k + p.wl.H + 1], p.uref, None, p.u_out, p.x_out)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(p.stream)
                evs[i] = (ev_start, ev)
                p.running = (i, ev, time.perf_counter() - t0)
                running.append(p)
            if not running and nxt < len(order):
                wait = arrivals[order[nxt]][0] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
        wall = time.perf_counter() - t0
        torch.cuda.synchronize(self.device)
        self.device_intervals = [(ev0.elapsed_time(a), ev0.elapsed_time(b)) for a, b in evs]
        return rec, outs, wall


def max_overlap(intervals):
    """Largest number of intervals (start, end) open at one instant."""
    pts = sorted([(s, 1) for s, _ in intervals] + [(e, -1) for _, e in intervals], key=lambda x: (x[0], x[1]))
    cur = best = 0
    for _, d in pts:
        cur += d
        best = max(best, cur)
    return best


def poisson_arrivals(rate, count, n_problems, seed):
    """`count` request times of a Poisson process of the given rate, each for
    a problem drawn uniformly."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    pid = rng.integers(0, n_problems, size=count)
    return [(float(a), int(b)) for a, b in zip(t, pid)]

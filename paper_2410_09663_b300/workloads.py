"""Seeded synthetic workloads for Kalman-MPC (arXiv 2410.09663).

This module only draws inputs: CNN weights, the input matrix B, the initial
field, reference fields and the random numbers the method consumes (W0, W, V).
It holds none of the method's arithmetic, and both the CUDA path and the FP64
oracle receive exactly the float32 values it produces.

The paper controls a PhyCRNet-style CNN trained on the 2-D Burgers' equation
(Numerical Experiments section); neither that network nor its data is
available, so every workload here is synthetic and stands in for it:

  * CNN_theta: input channels [X; B U], 3x3 "same" convolutions, tanh after
    hidden layers, one linear output channel, residual X + 0.1 * out.
    Each layer's 3x3 kernel from input channel i to output channel o is
        w[o][i] = sign * S / C_in + N(0, 0.01^2),
        S = [[0, 1/8, 0], [1/8, 1/2, 1/8], [0, 1/8, 0]] = I + L/8,
    with L the 5-point discrete Laplacian, sign = +1 for hidden layers and -1
    for the last layer, biases 0.  (I + L/8 is the explicit diffusion stencil
    built from the Laplacian; composing bare Laplacians through several layers
    with the 0.1 residual is unstable, so this stable reading is used.  The
    linearised surrogate relaxes X toward -B U: controllable and smooth.)
  * B ~ N(0, 0.1^2), n x l.
  * X_0 = centred Gaussian bump (amplitude 1, sigma = n/8) + N(0, 0.01^2).
  * reference: zero (small case) or two Gaussian blobs (amplitude 1) moving on
    opposite sides of a circle of radius n/4 about the centre with a period of
    50 control steps; U^ref = 0.
  * noise: W0, W ~ N(0, sigma_w^2), V_X ~ N(0, sigma_vx^2), V_U ~ N(0, sigma_vu^2),
    all 0.01, drawn per control step k from a generator keyed by (seed, k).
  * constraints (optional): a box |U| <= u_max on every control entry as 2 l
    affine rows (Gx = 0, Gu = [I; -I], h = u_max), softplus barrier alpha = 10,
    beta = 100 and eps ~ N(0, 0.01^2) drawn from its own generator keyed by
    (seed, k), so the other noise of a step is the same with or without it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SIGMA = 0.01

_PURPOSE = {"weights": 1, "B": 2, "X0": 3, "noise": 4, "generic": 5, "cnoise": 6}


def _rng(seed: int, purpose: str, *extra: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), _PURPOSE[purpose], *[int(e) for e in extra]])


@dataclass
class Constraints:
    """Inputs of c virtual constraint observations z = phi(Gx X + Gu U - h) +
    eps (reference 0, phi(x) = ln(1 + e^{beta x}) / alpha, eps ~ N(0, sigma_z^2))."""
    Gx: np.ndarray                    # c x n, float32
    Gu: np.ndarray                    # c x l, float32
    h: np.ndarray                     # c, float32
    alpha: float = 10.0
    beta: float = 100.0
    sigma_z: float = SIGMA

    @property
    def c(self):
        return int(self.h.size)


def u_box(n: int, l: int, u_max: float, alpha: float = 10.0, beta: float = 100.0, sigma_z: float = SIGMA):
    """|U[b][j]| <= u_max for every control entry: rows U - u_max and -U - u_max."""
    Gu = np.concatenate([np.eye(l), -np.eye(l)]).astype(np.float32)
    return Constraints(np.zeros((2 * l, n), np.float32), Gu, np.full(2 * l, u_max, np.float32), alpha, beta,
                       sigma_z)


@dataclass
class Workload:
    """Sizes and synthetic inputs of one Kalman-MPC problem."""
    name: str
    n: int
    m: int
    l: int
    channels: list
    N: int
    H: int
    S: int
    ref: str = "zero"                 # "zero" or "blobs"
    blob_sigma: float = 6.0
    residual_scale: float = 0.1
    sigma_w: float = SIGMA
    sigma_vx: float = SIGMA
    sigma_vu: float = SIGMA
    seed: int = 0
    extra: dict = field(default_factory=dict)
    cons: Constraints | None = None

    @property
    def q(self):
        return self.n + 2 * self.l

    @property
    def c(self):
        return self.cons.c if self.cons is not None else 0

    @property
    def p(self):
        return self.n + self.l + self.c

    @property
    def n_layers(self):
        return len(self.channels) - 1

    # ---------------------------------------------------------------- weights
    def weights(self):
        """List of (w [Cout][Cin][3][3] float32, b [Cout] float32)."""
        rng = _rng(self.seed, "weights")
        S = np.array([[0.0, 0.125, 0.0], [0.125, 0.5, 0.125], [0.0, 0.125, 0.0]])
        out = []
        L = self.n_layers
        for k in range(L):
            cin, cout = self.channels[k], self.channels[k + 1]
            sign = -1.0 if k == L - 1 else 1.0
            w = sign * S[None, None] / cin + rng.normal(0.0, 0.01, size=(cout, cin, 3, 3))
            b = np.zeros(cout)
            out.append((w.astype(np.float32), b.astype(np.float32)))
        return out

    def flat_weights(self):
        ws = self.weights()
        w = np.concatenate([a.ravel() for a, _ in ws]).astype(np.float32)
        b = np.concatenate([c.ravel() for _, c in ws]).astype(np.float32)
        return w, b

    def B(self):
        return _rng(self.seed, "B").normal(0.0, 0.1, size=(self.n, self.l)).astype(np.float32)

    # ------------------------------------------------------------------ fields
    def X0(self):
        n, m = self.n, self.m
        y, x = np.mgrid[0:n, 0:m].astype(np.float64)
        s = n / 8.0
        bump = np.exp(-(((y - (n - 1) / 2) ** 2) + ((x - (m - 1) / 2) ** 2)) / (2 * s * s))
        return (bump + _rng(self.seed, "X0").normal(0.0, 0.01, size=(n, m))).astype(np.float32)

    def U_init(self):
        return np.zeros((self.l, self.m), np.float32)

    def U_ref(self):
        return np.zeros((self.l, self.m), np.float32)

    def X_ref(self, k: int):
        """Reference field at absolute control time k."""
        n, m = self.n, self.m
        if self.ref == "zero":
            return np.zeros((n, m), np.float32)
        y, x = np.mgrid[0:n, 0:m].astype(np.float64)
        th = 2.0 * np.pi * k / 50.0
        r = n / 4.0
        cy, cx = (n - 1) / 2.0, (m - 1) / 2.0
        f = np.zeros((n, m))
        for sgn in (1.0, -1.0):
            py, px = cy + sgn * r * np.sin(th), cx + sgn * r * np.cos(th)
            f += np.exp(-(((y - py) ** 2) + ((x - px) ** 2)) / (2 * self.blob_sigma ** 2))
        return f.astype(np.float32)

    def X_ref_window(self, k: int):
        """References for times k .. k+H, shape (H+1, n, m)."""
        return np.stack([self.X_ref(k + s) for s in range(self.H + 1)])

    def X_ref_all(self, S: int | None = None):
        S = self.S if S is None else S
        return np.stack([self.X_ref(t) for t in range(S + self.H + 1)])

    # ------------------------------------------------------------------- noise
    def noise_floats(self):
        n, m, l, N, H = self.n, self.m, self.l, self.N, self.H
        return N * l * m + H * N * (l * m + n * m + l * m + self.c * m)

    def noise(self, k: int):
        """Random numbers of the solve at control step k, float32, laid out as
        W0 [N][l][m], W [H][N][l][m], V_X [H][N][n][m], V_U [H][N][l][m], then
        with constraints eps [H][N][c][m]."""
        n, m, l, N, H = self.n, self.m, self.l, self.N, self.H
        rng = _rng(self.seed, "noise", k)
        w0 = rng.standard_normal((N, l, m)) * self.sigma_w
        w = rng.standard_normal((H, N, l, m)) * self.sigma_w
        vx = rng.standard_normal((H, N, n, m)) * self.sigma_vx
        vu = rng.standard_normal((H, N, l, m)) * self.sigma_vu
        parts = [w0.ravel(), w.ravel(), vx.ravel(), vu.ravel()]
        if self.c:
            parts.append(_rng(self.seed, "cnoise", k).standard_normal((H, N, self.c, m)).ravel() * self.cons.sigma_z)
        return np.concatenate(parts).astype(np.float32)

    def noise_all(self, S: int | None = None):
        S = self.S if S is None else S
        return np.stack([self.noise(k) for k in range(S)])

    def with_(self, **kw):
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


def small_16():
    """16 x 16 field, l = 4, CNN 2 -> 8 -> 1, N = 32, H = 5, 10 control steps,
    zero reference."""
    return Workload("oic_16x16_N32_H5", n=16, m=16, l=4, channels=[2, 8, 1], N=32, H=5, S=10,
                    ref="zero")


def working_64():
    """64 x 64 field, l = 8, CNN 2 -> 32 -> 32 -> 1, N = 256, H = 10, 50 control
    steps, two moving blobs (sigma 6 px)."""
    return Workload("oic_64x64_N256_H10", n=64, m=64, l=8, channels=[2, 32, 32, 1], N=256, H=10,
                    S=50, ref="blobs", blob_sigma=6.0)


def large_128():
    """128 x 128 field, l = 16, CNN 2 -> 64 -> 64 -> 64 -> 1, N = 1024, H = 20,
    50 control steps, two moving blobs (sigma 12 px)."""
    return Workload("oic_128x128_N1024_H20", n=128, m=128, l=16, channels=[2, 64, 64, 64, 1],
                    N=1024, H=20, S=50, ref="blobs", blob_sigma=12.0)


def mix64(seed: int = 2024, count: int = 64):
    """Batched uneven problems: `count` independent problems with grids drawn
    uniformly from {32, 64, 96, 128}^2 (n = m), l = m / 8, N uniformly from
    {64, 128, 256, 512} and H uniformly from 5..20; CNN 2-32-32-1; each
    problem its own seed (weights, B, initial field, noise) and moving-blob
    reference (sigma m / 10)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.choice([32, 64, 96, 128]))
        N = int(rng.choice([64, 128, 256, 512]))
        H = int(rng.integers(5, 21))
        out.append(Workload(f"mix{i}_{m}x{m}_N{N}_H{H}", n=m, m=m, l=m // 8, channels=[2, 32, 32, 1], N=N, H=H,
                            S=50, ref="blobs", blob_sigma=m / 10.0, seed=seed + 1 + i))
    return out


WORKLOADS = {"small_16": small_16, "working_64": working_64, "large_128": large_128}
BATCHES = {"mix64": mix64}


# ------------------------------------------------------------------ Philox
# Counter-based generator Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
# written from its published definition; the CUDA library implements the same
# definition independently for its on-device noise mode.  Element e of a
# solve's noise buffer takes word e % 4 of the block for counter
# (e // 4 low, e // 4 high, solve low, solve high) under key (seed low, seed
# high); words become uniforms ((w >> 8) + 1/2) 2^-24 and pairs of uniforms
# become normals by Box-Muller.
_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: uint32 array (..., 4); key: (k0, k1) ints.  Returns uint32 (..., 4)."""
    c0, c1, c2, c3 = (ctr[..., i].astype(np.uint64) for i in range(4))
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def philox_normals(count: int, seed: int, solve: int):
    q = np.arange((count + 3) // 4, dtype=np.uint64)
    ctr = np.stack([q & _MASK, q >> np.uint64(32),
                    np.full_like(q, solve & 0xFFFFFFFF), np.full_like(q, (solve >> 32) & 0xFFFFFFFF)],
                   axis=-1).astype(np.uint32)
    w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    u = ((w >> 8).astype(np.float64) + 0.5) * (1.0 / 16777216.0)
    r0 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r1 = np.sqrt(-2.0 * np.log(u[:, 2]))
    z = np.stack([r0 * np.cos(2 * np.pi * u[:, 1]), r0 * np.sin(2 * np.pi * u[:, 1]),
                  r1 * np.cos(2 * np.pi * u[:, 3]), r1 * np.sin(2 * np.pi * u[:, 3])], axis=-1)
    return z.reshape(-1)[:count]


def philox_noise(wl: Workload, solve: int, seed: int | None = None):
    """The noise buffer the device draws for solve number `solve` (counted from
    the last reset) in Philox mode, same layout as Workload.noise."""
    seed = wl.seed if seed is None else seed
    n, m, l, N, H = wl.n, wl.m, wl.l, wl.N, wl.H
    z = philox_normals(wl.noise_floats(), seed, solve)
    e0 = N * l * m
    e1 = e0 + H * N * l * m
    e2 = e1 + H * N * n * m
    sig = np.empty_like(z)
    sig[:e1] = np.float32(wl.sigma_w)
    sig[e1:e2] = np.float32(wl.sigma_vx)
    e3 = e2 + H * N * l * m
    sig[e2:e3] = np.float32(wl.sigma_vu)
    if wl.c:
        sig[e3:] = np.float32(wl.cons.sigma_z)
    return (sig.astype(np.float32) * z.astype(np.float32)).astype(np.float32)

"""Seeded synthetic inputs for the spectral-deflation active-set workloads.

This module is shared by the CUDA path, the CPU oracle and the tests.  It only
draws random inputs (instance parameters mu and coefficient fields) and names
the workload shapes; it holds none of the method's arithmetic (no operator, no
desired-state evaluation, no solver).

Workloads (grid, operator, parameter law, instance count, number of modes k):

  ``diff2d_32``        32x32 interior grid, kappa = 1, alpha = 1e-4, psi = 1,
                       y_d = a exp(-|x-c|^2/(2*0.1^2)), a ~ U[1,3],
                       c ~ U[0.25,0.75]^2, 20 instances, k = 16.
  ``block2d_1024``     1024x1024, piecewise-constant kappa on 4x4 equal blocks
                       with log10 kappa ~ U[-1,1] (one draw shared by all
                       instances), same y_d law, 64 instances, k = 64.
  ``convdiff2d_512``   512x512, A = eps(-Laplace) + upwind(b), eps = 1e-2,
                       b = (cos theta, sin theta), theta ~ U[0, 2 pi),
                       a ~ U[1,4], 256 instances in one batch, k = 48.
  ``lognormal2d_2048`` 2048x2048, log kappa a zero-mean Gaussian field with
                       exponential covariance exp(-r/0.1) and sigma = 1 (one
                       draw), 32 instances, k = 128.
  ``diff3d_128``       128^3, kappa = 1, mu = (a, cx, cy, cz), a ~ U[1,3],
                       c ~ U[0.25,0.75]^3, 2000 training + 1024 held-out
                       instances, evaluated in batches of 128, k = 60.
  ``spacetime2d_64``   the all-at-once parabolic problem on a 64^2 spatial
                       grid with n_t = 16 implicit Euler steps on (0, 1]
                       (N = 65,536), kappa = 1, y_d ramped in time with
                       tau = 0.2, sigma = 0.12, a ~ U[1,3],
                       c ~ U[0.25,0.75]^2, 32 instances; k = 8 spatial modes,
                       Kronecker basis of rank 8 n_t = 128.

Every generator takes an explicit seed (numpy PCG64).  Parameters are drawn in
the order a, c, theta for each instance, instance by instance.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    n: int
    k: int
    instances: int
    a_range: tuple = (1.0, 3.0)
    c_range: tuple = (0.25, 0.75)
    sigma: float = 0.1          # width of the Gaussian desired state
    alpha: float = 1e-4
    psi: float = 1.0
    kappa: str = "const"        # "const" | "block4" | "lognormal"
    diff_scale: float = 1.0
    convection: bool = False
    batch: int = 1
    seed: int = 20260
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.n ** self.dim


WORKLOADS = {
    "diff2d_32": Workload("diff2d_32", 2, 32, 16, 20, seed=20260, batch=20),
    "block2d_1024": Workload("block2d_1024", 2, 1024, 64, 64, kappa="block4", seed=20261),
    "convdiff2d_512": Workload("convdiff2d_512", 2, 512, 48, 256, a_range=(1.0, 4.0),
                               diff_scale=1e-2, convection=True, batch=256, seed=20262),
    "lognormal2d_2048": Workload("lognormal2d_2048", 2, 2048, 128, 32, kappa="lognormal",
                                 seed=20263),
    "diff3d_128": Workload("diff3d_128", 3, 128, 60, 3024, batch=128, seed=20264,
                           extra={"train": 2000, "held_out": 1024}),
    "spacetime2d_64": Workload("spacetime2d_64", 2, 64, 8, 32, sigma=0.12, batch=32, seed=20265,
                               extra={"n_t": 16, "t_final": 1.0, "ramp_tau": 0.2}),
}


def scaled(w: Workload, n: int, **kw) -> Workload:
    """The same workload law on an n^dim grid (for parity cases that the
    oracle finishes in seconds)."""
    from dataclasses import replace
    return replace(w, n=n, name=f"{w.name}@{n}", **kw)


@dataclass
class Instance:
    """One parameter instance: desired-state amplitude and centre, and (for the
    convection-diffusion workload) the convection velocity."""
    a: float
    c: tuple
    b: tuple = (0.0, 0.0, 0.0)


def draw_instances(w: Workload, count: int | None = None, seed: int | None = None,
                   offset: int = 0):
    """Draw ``count`` instances (default: all of the workload) from its seed.
    ``offset`` skips that many instances of the same stream first."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    total = w.instances if count is None else count
    out = []
    for i in range(offset + total):
        a = rng.uniform(*w.a_range)
        c = tuple(rng.uniform(*w.c_range, size=w.dim)) + (0.0,) * (3 - w.dim)
        b = (0.0, 0.0, 0.0)
        if w.convection:
            theta = rng.uniform(0.0, 2.0 * np.pi)
            b = (float(np.cos(theta)), float(np.sin(theta)), 0.0)
        if i >= offset:
            out.append(Instance(float(a), tuple(float(v) for v in c), b))
    return out


def instances_array(insts):
    """Pack instances as a float64 array [B, 7] = (a, cx, cy, cz, bx, by, bz)."""
    return np.array([[i.a, *i.c, *i.b] for i in insts], dtype=np.float64).reshape(-1, 7)


def kappa_field(w: Workload, seed: int | None = None):
    """Node diffusivity in x-fastest order, or None for kappa = 1."""
    rng = np.random.default_rng((w.seed if seed is None else seed) + 7919)
    n = w.n
    if w.kappa == "const":
        return None
    if w.kappa == "block4":
        logk = rng.uniform(-1.0, 1.0, size=(4,) * w.dim)
        # node j (0-based) sits at x = (j+1)/(n+1); block = floor(4x)
        blk = np.minimum((4 * (np.arange(n) + 1)) // (n + 1), 3)
        if w.dim == 2:
            lk = logk[blk[:, None], blk[None, :]]          # [y, x]
        else:
            lk = logk[blk[:, None, None], blk[None, :, None], blk[None, None, :]]
        return np.ascontiguousarray(10.0 ** lk, dtype=np.float64).reshape(-1)
    if w.kappa == "lognormal":
        return np.exp(gaussian_field_2d(n, 0.1, 1.0, rng)).reshape(-1)
    raise ValueError(w.kappa)


def gaussian_field_2d(n: int, ell: float, sigma: float, rng) -> np.ndarray:
    """Zero-mean stationary Gaussian field on the n x n interior nodes
    (spacing h = 1/(n+1)) with covariance sigma^2 exp(-r/ell), sampled by
    circulant embedding on a 2n x 2n periodic grid (negative embedding
    eigenvalues, if any, are clipped to zero)."""
    h = 1.0 / (n + 1)
    m = 2 * n
    lag = np.minimum(np.arange(m), m - np.arange(m)) * h
    r = np.sqrt(lag[:, None] ** 2 + lag[None, :] ** 2)
    cov = sigma**2 * np.exp(-r / ell)
    lam = np.maximum(np.fft.fft2(cov).real, 0.0)
    xi = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    f = np.fft.fft2(np.sqrt(lam / (m * m)) * xi)
    return np.ascontiguousarray(f.real[:n, :n])


def psi_vector(w: Workload) -> np.ndarray:
    return np.full(w.N, w.psi, dtype=np.float64)


# ---------------------------------------------------------------------------
# learned warm start: the input box and the seeded initial MLP parameters

WARM_WIDTHS = (4, 256, 256, 256, 64)


def input_box(w: Workload):
    """Lower and upper bounds of the MLP inputs (a, c_1 .. c_dim)."""
    lo = [w.a_range[0]] + [w.c_range[0]] * w.dim
    hi = [w.a_range[1]] + [w.c_range[1]] * w.dim
    return lo, hi


def mlp_init(widths=WARM_WIDTHS, seed: int = 7) -> np.ndarray:
    """Initial MLP parameters (FP32 flat vector, layout W_1, b_1, ..., W_L,
    b_L with W row-major out x in): W ~ N(0, 1/fan_in), b = 0."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(len(widths) - 1):
        fi, fo = widths[i], widths[i + 1]
        parts.append((rng.standard_normal((fo, fi)) / np.sqrt(fi)).ravel())
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)

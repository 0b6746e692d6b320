"""Seeded synthetic inputs for the solver workloads.

This module holds no arithmetic of the method: it only evaluates the
coefficient fields and right-hand sides at node coordinates that the caller
supplies (from whichever Shishkin mesh the caller built), and draws the
seeded random numbers.  Both the CUDA path's tests/benchmark and the CPU
oracle consume these arrays, so both sides always see identical inputs.

The paper's own experiments use analytic manufactured solutions (Sec. 3.3)
rather than a dataset; the workloads here follow the problem statement
(eq. 2D): -eps*Lap(u) - c.grad(u) + r*u = f on (0,1)^2, zero Dirichlet data,
with c1, c2 >= beta > 0 and r >= 0.

Arrays are float64, length (N-1)**2, x-fastest over the interior nodes:
k = (j-1)*(N-1) + (i-1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def interior_grid(x: np.ndarray, y: np.ndarray):
    """Interior node coordinates as flat x-fastest arrays."""
    X, Y = np.meshgrid(x[1:-1], y[1:-1], indexing="xy")
    return X.ravel(), Y.ravel()


def fourier_coeffs(seed: int, kmax: int = 4) -> np.ndarray:
    """a_kl ~ N(0,1), drawn row-major (k outer, l inner), kmax*kmax values."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((kmax, kmax))


def fourier_rhs(x, y, a: np.ndarray) -> np.ndarray:
    """f = sum_{k,l} a_kl sin(k pi x) sin(l pi y) on the interior nodes."""
    X, Y = interior_grid(x, y)
    f = np.zeros_like(X)
    kmax = a.shape[0]
    for k in range(1, kmax + 1):
        sx = np.sin(k * np.pi * X)
        for l in range(1, a.shape[1] + 1):
            f += a[k - 1, l - 1] * sx * np.sin(l * np.pi * Y)
    return f


def fields_quadratic(x, y, a: float = 1.0, b: float = 1.0):
    """c1 = 1 + a x^2, c2 = 1 + b y^2, r = 1 + x y (min c1 = min c2 = 1)."""
    X, Y = interior_grid(x, y)
    return 1.0 + a * X * X, 1.0 + b * Y * Y, 1.0 + X * Y


def fields_trig(x, y):
    """c1 = 1.5 + 0.5 sin(2 pi x y), c2 = 1.5 + 0.5 cos(pi x), r = 1."""
    X, Y = interior_grid(x, y)
    return 1.5 + 0.5 * np.sin(2 * np.pi * X * Y), 1.5 + 0.5 * np.cos(np.pi * X), np.ones_like(X)


@dataclass
class Problem:
    N: int
    eps: float
    c1: np.ndarray
    c2: np.ndarray
    r: np.ndarray
    f: np.ndarray
    sigma: float = 2.0
    beta: float = 1.0


def problem_fourier_quadratic(x, y, N, eps, seed=0, a=1.0, b=1.0) -> Problem:
    """Single-instance workload: quadratic convection, bilinear reaction,
    16 seeded Fourier modes as forcing (sigma = 2, beta = 1)."""
    c1, c2, r = fields_quadratic(x, y, a, b)
    return Problem(N, eps, c1, c2, r, fourier_rhs(x, y, fourier_coeffs(seed)))


def problem_fourier_trig(x, y, N, eps, seed=2) -> Problem:
    """Large-mesh workload: trigonometric convection, unit reaction."""
    c1, c2, r = fields_trig(x, y)
    return Problem(N, eps, c1, c2, r, fourier_rhs(x, y, fourier_coeffs(seed)))


def mms_exponential(x, y, eps):
    """Manufactured problem of Sec. 3.3, eq. (exponential_MMS): c1 = 2,
    c2 = 3, r = 1 and u = cos(pi x/2)(1 - e^{-2x/eps})(1-y)^3(1 - e^{-3y/eps});
    returns (f, u) at the interior nodes, f = -eps Lap u - 2 u_x - 3 u_y + u
    written out by the product rule."""
    X, Y = interior_grid(x, y)
    ex, ey = np.exp(-2.0 * X / eps), np.exp(-3.0 * Y / eps)
    a, a1, a2 = np.cos(np.pi * X / 2), -np.pi / 2 * np.sin(np.pi * X / 2), -np.pi ** 2 / 4 * np.cos(np.pi * X / 2)
    b, b1, b2 = 1.0 - ex, 2.0 / eps * ex, -4.0 / eps ** 2 * ex
    c, c1, c2 = (1.0 - Y) ** 3, -3.0 * (1.0 - Y) ** 2, 6.0 * (1.0 - Y)
    d, d1, d2 = 1.0 - ey, 3.0 / eps * ey, -9.0 / eps ** 2 * ey
    Xf, Xf1, Xf2 = a * b, a1 * b + a * b1, a2 * b + 2 * a1 * b1 + a * b2
    Yf, Yf1, Yf2 = c * d, c1 * d + c * d1, c2 * d + 2 * c1 * d1 + c * d2
    u = Xf * Yf
    f = -eps * (Xf2 * Yf + Xf * Yf2) - 2.0 * Xf1 * Yf - 3.0 * Xf * Yf1 + u
    return f, u


def mms_parabolic(x, y, eps):
    """Manufactured problem of Sec. 3.3, eq. (parabolic_MMS): c1 = 1, c2 = 0,
    r = 1 and u = X(x) Y(y) with
        X = cos(pi x/2) - (e^{-x/eps} - e^{-1/eps}) / (1 - e^{-1/eps}),
        Y = (1 - e^{-y/sqrt(eps)}) / (1 - e^{-1/sqrt(eps)}) - y^{5/2};
    returns (f, u) at the interior nodes, f = -eps Lap u - u_x + u.  The
    1/eps terms of -eps X'' - X' cancel exactly and are left out:
        -eps X'' - X' = eps pi^2/4 cos(pi x/2) + pi/2 sin(pi x/2),
        -eps Y''      = e^{-y/sqrt(eps)} / (1 - e^{-1/sqrt(eps)}) + 15/4 eps sqrt(y)."""
    Xg, Yg = interior_grid(x, y)
    se = np.sqrt(eps)
    ex = np.exp(-Xg / eps)
    e1 = np.exp(-1.0 / eps)
    ey = np.exp(-Yg / se)
    e2 = np.exp(-1.0 / se)
    cx, sx_ = np.cos(np.pi * Xg / 2), np.sin(np.pi * Xg / 2)
    Xf = cx - (ex - e1) / (1.0 - e1)
    Yf = (1.0 - ey) / (1.0 - e2) - Yg ** 2.5
    u = Xf * Yf
    f = Yf * (eps * np.pi ** 2 / 4 * cx + np.pi / 2 * sx_) + Xf * (ey / (1.0 - e2) + 3.75 * eps * np.sqrt(Yg)) + u
    return f, u


def batch_params(count: int = 256, seed: int = 3, n_choices=tuple(range(64, 513, 32)),
                 log_eps=(-8.0, -2.0)):
    """Per-instance (N, eps, a, b, fourier seed) for the batched workload:
    N uniform over n_choices, log10(eps) uniform, a, b uniform in [0, 1]."""
    rng = np.random.default_rng(seed)
    Ns = rng.choice(np.asarray(n_choices), size=count)
    eps = 10.0 ** rng.uniform(log_eps[0], log_eps[1], size=count)
    a = rng.uniform(0.0, 1.0, size=count)
    b = rng.uniform(0.0, 1.0, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [dict(N=int(Ns[i]), eps=float(eps[i]), a=float(a[i]), b=float(b[i]), seed=int(seeds[i]))
            for i in range(count)]


def adjoint_batch(N: int, nrhs: int = 16, seed: int = 4):
    """Seeded Fourier coefficient sets for nrhs right-hand sides and the
    objective weights w ~ U[0,1] over the interior nodes."""
    rng = np.random.default_rng(seed)
    coeffs = [rng.standard_normal((4, 4)) for _ in range(nrhs)]
    w = rng.uniform(0.0, 1.0, size=(N - 1) ** 2)
    return coeffs, w

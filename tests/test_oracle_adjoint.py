"""Pins of the oracle's adjoint gradient against finite differences and a
dense adjoint: J = 1/2 sum_i w_i u_i^2 with A(c1, c2, r) u = f."""
import numpy as np

import oracle
from paper_2108_13468_gb300 import inputs


def _setup(N=16, eps=1e-3):
    x, _ = oracle.mesh(N, eps)
    y = x.copy()
    p = inputs.problem_fourier_quadratic(x, y, N, eps)
    coeffs, w = inputs.adjoint_batch(N, nrhs=1, seed=4)
    return x, y, p, w


def J_of(N, eps, x, y, c1, c2, r, f, w):
    A = oracle.assemble(N, eps, x, y, c1, c2, r)
    u = np.linalg.solve(oracle.dense(N, A), f)
    return 0.5 * np.sum(w * u * u)


def test_adjoint_gradient_vs_central_differences():
    N, eps = 16, 1e-3
    x, y, p, w = _setup(N, eps)
    A = oracle.assemble(N, eps, x, y, p.c1, p.c2, p.r)
    u = oracle.band_solve(N, A, p.f)
    lam = oracle.band_solve(N, A, w * u, transpose=True)       # A^T lam = dJ/du
    g1, g2, gr = oracle.grad(N, x, y, u, lam)
    grads = {"f": lam, "c1": g1, "c2": g2, "r": gr}
    rng = np.random.default_rng(5)
    base = dict(c1=p.c1, c2=p.c2, r=p.r, f=p.f)
    for name, g in grads.items():
        for _ in range(8):
            d = rng.standard_normal(g.size)
            d /= np.linalg.norm(d)
            h = 1e-6 * max(1.0, np.abs(base[name]).max())
            plus, minus = dict(base), dict(base)
            plus[name] = base[name] + h * d
            minus[name] = base[name] - h * d
            fd = (J_of(N, eps, x, y, plus["c1"], plus["c2"], plus["r"], plus["f"], w)
                  - J_of(N, eps, x, y, minus["c1"], minus["c2"], minus["r"], minus["f"], w)) / (2 * h)
            assert abs(fd - g @ d) <= 1e-6 * max(abs(fd), np.abs(g).max() * 1e-3), (name, fd, g @ d)


def test_adjoint_vs_dense_sensitivity():
    """dJ/dc1_k from the dense formula -lam^T (dA/dc1_k) u with dA/dc1_k read
    off the assembled matrix by differentiating its entries (complex step)."""
    N, eps = 8, 1e-2
    x, y, p, w = _setup(N, eps)
    A = oracle.assemble(N, eps, x, y, p.c1, p.c2, p.r)
    D = oracle.dense(N, A)
    u = np.linalg.solve(D, p.f)
    lam = np.linalg.solve(D.T, w * u)
    g1, g2, gr = oracle.grad(N, x, y, u, lam)
    n = (N - 1) ** 2
    for name, g in (("c1", g1), ("c2", g2), ("r", gr)):
        for k in (0, n // 2, n - 1, 5):
            pert = {"c1": p.c1.copy(), "c2": p.c2.copy(), "r": p.r.copy()}
            pert[name][k] += 1.0                 # A is affine in each field
            dD = oracle.dense(N, oracle.assemble(N, eps, x, y, pert["c1"], pert["c2"], pert["r"])) - D
            assert np.isclose(g[k], -lam @ dD @ u, rtol=1e-7, atol=1e-12 * np.abs(g).max())

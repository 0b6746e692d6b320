"""The oracle's graded layer mesh (the Remark after Theorem (big bound):
the theory also covers graded meshes; the Bakhvalov-Shishkin mesh of Linss
(1999) keeps the Shishkin transition point and the N/2 + N/2 split) against
what fixes it independently of its code:

* its generating identity, exp(-beta x_i / (sigma eps)) = 1 - 2 (1 - 1/N) i/N
  on the layer (the mesh samples the layer function uniformly), the
  transition node x_{N/2} = tau, uniform interior widths, graded layer
  widths, and the uniform mesh when tau is capped at 1/2;
* the convergence theory of upwind differences on such meshes: the error of
  the paper's exponential manufactured solution falls like N^-1 uniformly
  in eps, without the ln N factor of the Shishkin mesh, so its observed
  rate approaches 1 while the Shishkin rate stays near log2(2 ln N / ln 2N),
  and it is below the Shishkin error at every N.
"""
import numpy as np
import pytest

import oracle
from paper_2108_13468_gb300 import inputs


@pytest.mark.parametrize("N", [8, 64, 1024])
@pytest.mark.parametrize("eps,beta", [(1e-2, 1.0), (1e-4, 2.0), (1e-8, 3.0)])
def test_graded_mesh_nodes(N, eps, beta):
    sigma = 2.5
    x, tau = oracle.mesh(N, eps, sigma, beta, graded=True)
    xs, taus = oracle.mesh(N, eps, sigma, beta)
    m = N // 2
    assert tau == taus == min(0.5, sigma * eps * np.log(N) / beta)
    assert x[0] == 0.0 and x[m] == tau and x[N] == 1.0
    h = np.diff(x)
    assert np.all(h > 0)
    np.testing.assert_array_equal(x[m:], xs[m:])                     # interior part: the Shishkin nodes
    if tau < 0.5:
        i = np.arange(m)
        np.testing.assert_allclose(np.exp(-beta * x[:m] / (sigma * eps)), 1.0 - 2.0 * (1.0 - 1.0 / N) * i / N,
                                   rtol=1e-13, atol=0)
        assert np.all(np.diff(h[:m]) > 0)                               # widths grow through the layer
        assert h[0] < tau / m < h[m - 1]                                # finer than Shishkin at the wall


def test_graded_mesh_capped_tau_is_uniform():
    x, tau = oracle.mesh(16, 0.3, 2.0, 1.0, graded=True)
    assert tau == 0.5
    np.testing.assert_allclose(x, np.linspace(0.0, 1.0, 17), rtol=0, atol=1e-15)


def mms_error(N, eps, graded):
    x, _ = oracle.mesh(N, eps, 2.5, 2.0, graded=graded)
    y, _ = oracle.mesh(N, eps, 2.5, 3.0, graded=graded)
    f, ue = inputs.mms_exponential(x, y, eps)
    one = np.ones_like(f)
    A = oracle.assemble(N, eps, x, y, 2.0 * one, 3.0 * one, one)
    return float(np.abs(oracle.band_solve(N, A, f) - ue).max())


def test_graded_mesh_first_order_without_log_factor():
    eps = 1e-6
    Ns = (64, 128, 256)
    eg = [mms_error(N, eps, True) for N in Ns]
    es = [mms_error(N, eps, False) for N in Ns]
    rg = [np.log2(eg[k] / eg[k + 1]) for k in range(2)]
    rs = [np.log2(es[k] / es[k + 1]) for k in range(2)]
    assert all(g < s for g, s in zip(eg, es))
    assert rg[1] >= 0.95 and rg[0] < rg[1] <= 1.02          # approaching 1 from below
    assert rs[1] <= log_rate(128) + 0.02                      # Shishkin: N^-1 ln N
    # eps-uniform: the same error at a much smaller eps
    assert abs(mms_error(128, 1e-8, True) - eg[1]) <= 1e-2 * eg[1]


def log_rate(N):
    return float(np.log2(2.0 * np.log(N) / np.log(2 * N)))

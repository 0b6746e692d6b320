"""The general Shishkin mesh on the GPU (the Remark on general Shishkin
meshes): NL = qN intervals in the layer, tau = min(q, sigma eps ln N / beta),
and the blocks of Sec. 3.1 split at layer index NL (blp_params.
layer_intervals).  Against the oracle on the same split:

* the preconditioner z = (D^-1 M)^-1 v = M^-1 (D v) to 1e-11 in FP64 with the
  same corner cycle count, and within the FP32 bound at fixed cycles;
* solves to 1e-8 (FP64) / 1e-7 (mixed) of the banded-LU solution;
* layer shares below and above 1/2, an odd layer count (a corner that does
  not coarsen), and N = 1024 with q = 1/4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2108_13468_gb300 as blp  # noqa: E402
from paper_2108_13468_gb300 import _native, inputs  # noqa: E402


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    a = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def problem(N, NL, eps, seed=0):
    x, _ = oracle.mesh(N, eps, layer_intervals=NL)
    p = inputs.problem_fourier_quadratic(x, x, N, eps, seed=seed)
    return x, p, oracle.assemble(N, eps, x, x, p.c1, p.c2, p.r)


CASES = [(64, 16, 1e-4), (128, 96, 1e-6), (130, 40, 1e-2), (96, 33, 1e-8)]


@pytest.mark.parametrize("N,NL,eps", CASES)
@pytest.mark.parametrize("fixed", [0, 2])
def test_general_split_preconditioner(N, NL, eps, fixed):
    x, p, A = problem(N, NL, eps)
    P = oracle.Prec(N, eps, x, x, p.c1, p.c2, p.r, fixed_cycles=fixed, layer_intervals=NL)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), layer_intervals=NL, corner_fixed_cycles=fixed)
    v = np.random.default_rng(2).standard_normal((N - 1) ** 2)
    zo, co = P.apply(A["C"] * v)
    z, c = s.precond(T(v))
    assert c == co and rel(z, zo) < 1e-11, (c, co, rel(z, zo))
    zto, cto = P.apply(v, transpose=True)
    zt, ct = s.precond(T(v), transpose=True)
    assert ct == cto and rel(zt, A["C"] * zto) < 1e-11
    if fixed:
        assert rel(s.precond(T(v), precision=blp.BLP_MIXED)[0], zo) < 1e-4
    s.close()


@pytest.mark.parametrize("N,NL,eps", CASES)
@pytest.mark.parametrize("precision,tol", [(blp.BLP_FP64, 1e-8), (blp.BLP_MIXED, 1e-7)])
def test_general_split_solve_matches_direct(N, NL, eps, precision, tol):
    x, p, A = problem(N, NL, eps, seed=1)
    ue = oracle.band_solve(N, A, p.f)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), layer_intervals=NL, precision=precision, maxit=3000)
    u, info = s.solve(T(p.f), tol=1e-10)
    s.close()
    assert info.status == 0 and info.relres <= 1e-10
    assert rel(u, ue) <= tol


def test_general_split_n1024_against_oracle_fgmres():
    """N = 1024, q = 1/4: the oracle's FGMRES on the same split at 1e-13
    stands in for the direct solve (banded LU needs ~17 GB here)."""
    N, NL, eps = 1024, 256, 1e-6
    x, p, A = problem(N, NL, eps, seed=1)
    P = oracle.Prec(N, eps, x, x, p.c1, p.c2, p.r, layer_intervals=NL)
    uo, st, it, rr, mc = oracle.fgmres(N, A, p.f, P, tol=1e-13)
    assert st == 0
    for precision, tol in ((blp.BLP_FP64, 1e-8), (blp.BLP_MIXED, 1e-7)):
        s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), layer_intervals=NL, precision=precision)
        u, info = s.solve(T(p.f), tol=1e-10)
        s.close()
        assert info.status == 0 and rel(u, uo) <= tol, (precision, rel(u, uo))


def test_general_split_arguments():
    N, eps = 64, 1e-4
    x, p, _ = problem(N, 16, eps)
    args = (T(p.c1), T(p.c2), T(p.r))
    for bad in (dict(layer_intervals=N - 1), dict(layer_intervals=-2),
                dict(layer_intervals=16, mesh=blp.BLP_MESH_GRADED)):
        with pytest.raises(blp.BlpError) as e:
            blp.Solver(N, eps, *args, **bad)
        assert e.value.status == _native.BLP_ERR_ARG
    s = blp.Solver(N, eps, *args, layer_intervals=N // 2)   # N/2: the mesh of Sec. 3
    s.close()

"""Paper-faithful mode on the GPU (Sec. 3.3): the manufactured problem of eq.
(exponential_MMS) with the paper's 2D mesh constants (sigma = 5/2, C1 = 2,
C2 = 3), solved through the C ABI.

* Table tab:exponential_errors: the maximum-norm error of the converged GPU
  solution against the manufactured solution, every printed entry up to
  N = 2048 within 1% (the oracle's exact discrete solution reproduces the
  entries it can reach, N <= 256, to the same 1%).
* Table tab:exponential_times_iters: FGMRES iteration counts under the
  paper's stopping rule ||f - A u||_2 <= 10 N^-1 ln N (FGMRES on A itself,
  as the paper), within one iteration of the printed count at N <= 256 and
  two at N = 512, 1024 (the GPU orthogonalises by CGS2, the paper by MGS).
  At N = 2048 the printed counts for eps <= 1e-6 are below what the method
  gives as read here (the oracle takes 8 at eps = 1e-6, where the table
  prints 5, and does not reach the absolute target at eps = 1e-7, the FP64
  floor of the unscaled residual there); at that size the FP64 GPU count is
  checked against the oracle's own count instead.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_13468_gb300 as blp  # noqa: E402
from paper_2108_13468_gb300 import inputs  # noqa: E402
from tests.conftest import read_table  # noqa: E402

NS = (128, 256, 512, 1024, 2048)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def mms_solver(N, eps, **params):
    x, _ = blp.mesh(N, eps, 2.5, 2.0)
    y, _ = blp.mesh(N, eps, 2.5, 3.0)
    f, ue = inputs.mms_exponential(x, y, eps)
    one = np.ones_like(f)
    s = blp.Solver(N, eps, T(2.0 * one), T(3.0 * one), T(one), sigma=2.5, beta_x=2.0, beta_y=3.0,
                   maxit=500, **params)
    return s, f, ue


def test_exponential_error_table():
    header, rows = read_table("table_exponential_errors.txt")
    for eps_s, vals in rows.items():
        eps = float(eps_s)
        for N, ref in zip(NS, vals):
            s, f, ue = mms_solver(N, eps, precision=blp.BLP_FP64)
            u, info = s.solve(T(f), tol=1e-12)
            s.close()
            assert info.status == 0
            err = float(np.abs(u.cpu().numpy() - ue).max())
            assert abs(err - ref) <= 0.01 * ref, (eps, N, err, ref)


def test_exponential_iteration_table():
    """The paper computes in double precision: the faithful mode is FP64."""
    header, rows = read_table("table_exponential_iterations.txt")
    for eps_s, vals in rows.items():
        eps = float(eps_s)
        for N, ref in zip(NS[:4], vals[:4]):
            s, f, ue = mms_solver(N, eps, precision=blp.BLP_FP64, stop_mode=blp.BLP_STOP_ABS2, restart=64)
            u, info = s.solve(T(f), tol=10.0 * np.log(N) / N)
            s.close()
            assert info.status == 0
            slack = 1 if N <= 256 else 2
            assert abs(info.iters - int(ref)) <= slack, (eps, N, info.iters, ref)


def test_mixed_precision_under_the_paper_rule():
    """The mixed path keeps Arnoldi on D^-1 A and checks the paper's
    absolute residual between restarts; it meets the rule.  (Under the
    default scaled rule the mixed and FP64 iteration counts agree.)"""
    header, rows = read_table("table_exponential_iterations.txt")
    for eps_s, vals in rows.items():
        eps = float(eps_s)
        for N, ref in zip(NS[:4], vals[:4]):
            s, f, ue = mms_solver(N, eps, precision=blp.BLP_MIXED, stop_mode=blp.BLP_STOP_ABS2, restart=64)
            u, info = s.solve(T(f), tol=10.0 * np.log(N) / N)
            s.close()
            assert info.status == 0 and info.relres <= 10.0 * np.log(N) / N, (eps, N, info.relres)


def test_exponential_iterations_n2048_match_oracle():
    import oracle
    N = 2048
    for eps in (1e-4, 1e-5, 1e-6):
        x, _ = oracle.mesh(N, eps, 2.5, 2.0)
        y, _ = oracle.mesh(N, eps, 2.5, 3.0)
        f, ue = inputs.mms_exponential(x, y, eps)
        one = np.ones_like(f)
        A = oracle.assemble(N, eps, x, y, 2.0 * one, 3.0 * one, one)
        P = oracle.Prec(N, eps, x, y, 2.0 * one, 3.0 * one, one)
        _, st, it_o, rr, mc = oracle.fgmres(N, A, f, P, tol=10.0 * np.log(N) / N, tol_abs=True, scaled=False,
                                            restart=100, maxit=80)
        assert st == 0
        s, f2, _ = mms_solver(N, eps, precision=blp.BLP_FP64, stop_mode=blp.BLP_STOP_ABS2, restart=64)
        u, info = s.solve(T(f2), tol=10.0 * np.log(N) / N)
        s.close()
        assert info.status == 0 and abs(info.iters - it_o) <= 1, (eps, info.iters, it_o)

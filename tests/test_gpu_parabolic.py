"""One parabolic and one exponential layer on the GPU (BLP_MESH_PARABOLIC):
the mesh of eq. (tau parabolic) in y, the blocks of Sec. 3.1 and the corner
cycle of Sec. 3.2 for this case (x-semicoarsening, operator-induced
interpolation, Galerkin coarse levels, downstream Gauss-Seidel, a 10^2
reduction), against the oracle:

* (the library's parabolic mesh equals the oracle's node for node:
  tests/test_abi.py, on the CPU);
* the preconditioner z = (D^-1 M)^-1 v = M^-1 (D v) matches the oracle's
  (oracle.Prec(parabolic=True)) to 1e-11 in FP64 with the same corner cycle
  count, and within the FP32 bound in mixed precision at fixed cycles;
* solves match the oracle's banded LU (FP64 1e-8, mixed 1e-7);
* the paper's problem (eq. parabolic_MMS, sigma = 5/2, C_low = 1) under the
  paper's stop: every entry of tab:parabolic_errors up to N = 2048 within
  1%, the counts of tab:parabolic_times_iters exactly for eps = 1e-5 and
  1e-6 (N = 128 ... 2048), within one of the oracle's count at N <= 512 for
  every eps, and corner solves of at most 3 V-cycles;
* adjoint solves and transposed applications are refused (the cycle is
  defined forward only).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2108_13468_gb300 as blp  # noqa: E402
from paper_2108_13468_gb300 import _native, inputs  # noqa: E402
from tests.conftest import read_table  # noqa: E402

NS = (128, 256, 512, 1024, 2048)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    a = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def meshes(N, eps, sigma=2.0, beta=1.0):
    x, _ = oracle.mesh(N, eps, sigma, beta)
    y, _ = oracle.mesh(N, eps, sigma, 1.0, parabolic=True)
    return x, y


def field_problem(N, eps, seed=0):
    """Variable fields with c2 >= 0 and no y-convection bound: c1 = 1 + x^2,
    c2 = y^2 / 2 (zero on the wall y = 0), r = 1 + x y, Fourier forcing."""
    x, y = meshes(N, eps)
    X, Y = inputs.interior_grid(x, y)
    c1, c2, r = 1.0 + X * X, 0.5 * Y * Y, 1.0 + X * Y
    f = inputs.fourier_rhs(x, y, inputs.fourier_coeffs(seed))
    return x, y, c1, c2, r, f


def solver(N, eps, c1, c2, r, **kw):
    return blp.Solver(N, eps, T(c1), T(c2), T(r), mesh=blp.BLP_MESH_PARABOLIC, corner_reduction=1e2, **kw)


CASES = [(64, 1e-2), (128, 1e-5), (96, 1e-8), (130, 1e-6)]


@pytest.mark.parametrize("N,eps", CASES)
@pytest.mark.parametrize("fixed", [0, 3])
def test_parabolic_preconditioner(N, eps, fixed):
    x, y, c1, c2, r, _ = field_problem(N, eps)
    A = oracle.assemble(N, eps, x, y, c1, c2, r)
    P = oracle.Prec(N, eps, x, y, c1, c2, r, reduction=1e2, fixed_cycles=fixed, parabolic=True)
    s = solver(N, eps, c1, c2, r, corner_fixed_cycles=fixed)
    v = np.random.default_rng(2).standard_normal((N - 1) ** 2)
    zo, co = P.apply(A["C"] * v)
    z, c = s.precond(T(v))
    assert c == co and rel(z, zo) < 1e-11, (c, co, rel(z, zo))
    if fixed:   # FP32: same cycle count by construction
        assert rel(s.precond(T(v), precision=blp.BLP_MIXED)[0], zo) < 1e-4
    s.close()


@pytest.mark.parametrize("N,eps", CASES)
@pytest.mark.parametrize("precision,tol", [(blp.BLP_FP64, 1e-8), (blp.BLP_MIXED, 1e-7)])
def test_parabolic_solve_matches_direct(N, eps, precision, tol):
    x, y, c1, c2, r, f = field_problem(N, eps, seed=1)
    A = oracle.assemble(N, eps, x, y, c1, c2, r)
    ue = oracle.band_solve(N, A, f)
    s = solver(N, eps, c1, c2, r, precision=precision)
    u, info = s.solve(T(f), tol=1e-10)
    s.close()
    assert info.status == 0 and info.relres <= 1e-10
    assert rel(u, ue) <= tol
    un = u.cpu().numpy()
    res = (f - oracle.apply(N, A, un)) / A["C"]
    assert np.linalg.norm(res) <= 1.0001e-10 * np.linalg.norm(f / A["C"])


def mms_solver(N, eps, **kw):
    x, _ = blp.mesh(N, eps, 2.5, 1.0)
    y, _ = blp.mesh(N, eps, 2.5, parabolic=True)
    f, ue = inputs.mms_parabolic(x, y, eps)
    one = np.ones_like(f)
    s = blp.Solver(N, eps, T(one), T(0.0 * one), T(one), sigma=2.5, beta_x=1.0, mesh=blp.BLP_MESH_PARABOLIC,
                   corner_reduction=1e2, maxit=500, **kw)
    return s, f, ue


def paper_stop_solve(N, eps, precision=blp.BLP_FP64):
    """The paper's solve: FGMRES on A (FP64) stopped by ||f - A u||_2 <= 10 ln(N)/N."""
    s, f, ue = mms_solver(N, eps, precision=precision, stop_mode=blp.BLP_STOP_ABS2)
    u, info = s.solve(T(f), tol=10.0 * np.log(N) / N)
    s.close()
    return u, info, ue


def test_parabolic_error_table():
    """tab:parabolic_errors lists the error of the iterate the paper's stop
    returns: the GPU's iterate under the same stop is within 1% at every
    entry.  At eps = 1e-8, N = 2048 the FP64 rounding floor of the unscaled
    residual lies above the absolute target, so no FP64 run stops there; the
    converged solution (scaled tolerance 1e-12) is compared instead."""
    header, rows = read_table("table_parabolic_errors.txt")
    for eps_s, vals in rows.items():
        eps = float(eps_s)
        for N, ref in zip(NS, vals):
            if eps == 1e-8 and N == 2048:
                s, f, ue = mms_solver(N, eps, precision=blp.BLP_FP64)
                u, info = s.solve(T(f), tol=1e-12)
                s.close()
                assert info.corner_cycles_max == 3
            else:
                u, info, ue = paper_stop_solve(N, eps)
            assert info.status == 0, (eps, N)
            err = float(np.abs(u.cpu().numpy() - ue).max())
            assert abs(err - ref) <= 0.01 * ref, (eps, N, err, ref)


def test_parabolic_iteration_counts():
    """tab:parabolic_times_iters under the paper's stop (FGMRES on A, FP64):
    every count of the eps = 1e-5 and 1e-6 rows exactly, N = 128 ... 2048;
    at N <= 512 every eps within one of the oracle's count (CGS2 against
    MGS), and corner solves of at most the paper's 3 V-cycles."""
    header, rows = read_table("table_parabolic_iterations.txt")
    for eps_s in ("1e-5", "1e-6"):
        for N, ref in zip(NS, rows[eps_s]):
            _, info, _ = paper_stop_solve(N, float(eps_s))
            assert info.status == 0 and info.iters == int(ref), (eps_s, N, info.iters, ref)
    for eps_s, vals in rows.items():
        eps = float(eps_s)
        for N in NS[:3]:
            target = 10.0 * np.log(N) / N
            x, y = meshes(N, eps, 2.5, 1.0)
            f, _ = inputs.mms_parabolic(x, y, eps)
            one = np.ones_like(f)
            A = oracle.assemble(N, eps, x, y, one, 0.0 * one, one)
            P = oracle.Prec(N, eps, x, y, one, 0.0 * one, one, reduction=1e2, parabolic=True)
            _, st, it_o, _, mc = oracle.fgmres(N, A, f, P, tol=target, tol_abs=True, scaled=False)
            assert st == 0 and mc == 3
            _, info, _ = paper_stop_solve(N, eps)
            assert info.status == 0 and abs(info.iters - it_o) <= 1, (eps, N, info.iters, it_o)
            assert 1 <= info.corner_cycles_max <= 3


def test_parabolic_refuses_the_adjoint_and_transposed_applications():
    N, eps = 64, 1e-4
    x, y, c1, c2, r, f = field_problem(N, eps)
    s = solver(N, eps, c1, c2, r)
    with pytest.raises(blp.BlpError) as e:
        s.solve_adjoint(T(f))
    assert e.value.status == _native.BLP_ERR_ARG
    with pytest.raises(blp.BlpError):
        s.precond(T(f), transpose=True)
    u, info = s.solve(T(f), tol=1e-10)     # the handle still solves forward
    assert info.status == 0
    s.close()


def test_parabolic_coefficient_check():
    """c2 >= 0 is required (beta_y is not used), c1 >= beta_x still is."""
    N, eps = 32, 1e-4
    x, y, c1, c2, r, _ = field_problem(N, eps)
    solver(N, eps, c1, c2, r).close()                      # c2 = 0 on the wall: accepted
    with pytest.raises(blp.BlpError) as e:
        solver(N, eps, c1, c2 - 1e-3, r)
    assert e.value.status == _native.BLP_ERR_COEF
    with pytest.raises(blp.BlpError):
        solver(N, eps, 0.5 * c1, c2, r)

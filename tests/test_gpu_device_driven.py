"""The device-driven FGMRES: one CUDA graph per solve, whose conditional nodes
take every restart, iteration and corner-cycle decision of Sec. 3.3's
restarted FGMRES and Sec. 3.2's stationary corner iteration on the device
(blp_params.device_driven = 1).

It runs the same kernels in the same order as the host-driven loop (the
default), so the two must agree bit for bit: solution, iteration and
restart counts, largest corner cycle count.  Both are also checked against
the oracle's banded-LU solution at the stated tolerances (FP64 1e-8, mixed
1e-7).  Cases cover both precisions, forward and adjoint solves, the fused
single-kernel corner (small N), fixed corner cycles, restarts, the iteration
budget running out, the parabolic-layer corner cycle, and a graph replayed
for a second right-hand side on the same handle."""
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
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def problem(N, eps, seed=0):
    x, _ = oracle.mesh(N, eps)
    p = inputs.problem_fourier_quadratic(x, x, N, eps, seed=seed)
    return p, oracle.assemble(N, eps, x, x, p.c1, p.c2, p.r)


def run(monkeypatch, graph, N, eps, p, rhs, adjoint=False, **params):
    monkeypatch.delenv("BLP_SOLVE_GRAPH", raising=False)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), device_driven=int(graph), **params)
    try:
        fn = s.solve_adjoint if adjoint else s.solve
        out = []
        for f in rhs:
            u, info = fn(T(f), raise_on_noconv=False)
            out.append((u.cpu().numpy(), info))
        return out, s.kernel_launches()
    finally:
        s.close()


def same(d, h):
    (ud, id_), (uh, ih) = d, h
    assert id_.device_driven == 1 and ih.device_driven == 0
    assert (id_.status, id_.iters, id_.restarts, id_.corner_cycles_max) == \
        (ih.status, ih.iters, ih.restarts, ih.corner_cycles_max)
    assert id_.relres == ih.relres
    assert np.array_equal(ud, uh)


CASES = [
    (64, 1e-4, blp.BLP_FP64, {}),
    (96, 1e-2, blp.BLP_MIXED, {}),
    (128, 1e-8, blp.BLP_MIXED, {}),
    (128, 1e-6, blp.BLP_FP64, {"restart": 4}),       # several restart cycles
    (130, 1e-3, blp.BLP_FP64, {"corner_fixed_cycles": 2}),
    (10, 1e-6, blp.BLP_FP64, {}),                     # the whole corner iteration in one fused kernel
    (256, 1e-4, blp.BLP_MIXED, {"restart": 8}),
]


@pytest.mark.parametrize("N,eps,precision,extra", CASES)
@pytest.mark.parametrize("adjoint", [False, True])
def test_device_driven_equals_host_loop(monkeypatch, N, eps, precision, extra, adjoint):
    p, A = problem(N, eps)
    d, nd = run(monkeypatch, True, N, eps, p, [p.f], adjoint, precision=precision, **extra)
    h, nh = run(monkeypatch, False, N, eps, p, [p.f], adjoint, precision=precision, **extra)
    same(d[0], h[0])
    assert d[0][1].status == 0
    # the counts differ by the host path's skipped corner-cycle launches
    assert 0 < nd < 2 * nh
    ue = oracle.band_solve(N, A, p.f, transpose=adjoint)
    tol = 1e-8 if precision == blp.BLP_FP64 else 1e-7
    assert rel(d[0][0], ue) <= tol


@pytest.mark.parametrize("precision", [blp.BLP_FP64, blp.BLP_MIXED])
def test_parabolic_corner_cycle_on_the_device(monkeypatch, precision):
    """The fields of the parabolic-layer case (c2 >= 0, zero on y = 0)."""
    N, eps = 128, 1e-6
    x, _ = oracle.mesh(N, eps)
    y, _ = oracle.mesh(N, eps, 2.0, 1.0, parabolic=True)
    X, Y = inputs.interior_grid(x, y)

    class P:
        c1, c2, r = 1.0 + X * X, 0.5 * Y * Y, 1.0 + X * Y
        f = inputs.fourier_rhs(x, y, inputs.fourier_coeffs(2))
    p = P
    kw = dict(precision=precision, mesh=blp.BLP_MESH_PARABOLIC, corner_reduction=1e2)
    d, _ = run(monkeypatch, True, N, eps, p, [p.f], **kw)
    h, _ = run(monkeypatch, False, N, eps, p, [p.f], **kw)
    same(d[0], h[0])
    assert d[0][1].status == 0


def test_budget_runs_out_on_the_device(monkeypatch):
    N, eps = 128, 1e-2
    p, _ = problem(N, eps)
    for precision in (blp.BLP_FP64, blp.BLP_MIXED):
        d, _ = run(monkeypatch, True, N, eps, p, [p.f], precision=precision, restart=5, maxit=13)
        h, _ = run(monkeypatch, False, N, eps, p, [p.f], precision=precision, restart=5, maxit=13)
        same(d[0], h[0])
        assert d[0][1].status == _native.BLP_ERR_NOCONV and d[0][1].iters == 13 and d[0][1].restarts == 3


def test_graph_replayed_for_another_right_hand_side(monkeypatch):
    """The second solve on a handle replays the graph built by the first."""
    N, eps = 128, 1e-4
    p, A = problem(N, eps)
    x, _ = oracle.mesh(N, eps)
    f2 = inputs.problem_fourier_quadratic(x, x, N, eps, seed=7).f
    for precision in (blp.BLP_FP64, blp.BLP_MIXED):
        d, _ = run(monkeypatch, True, N, eps, p, [p.f, f2, p.f], precision=precision)
        h, _ = run(monkeypatch, False, N, eps, p, [p.f, f2], precision=precision)
        same(d[0], h[0])
        same(d[1], h[1])
        assert np.array_equal(d[2][0], d[0][0])
        tol = 1e-8 if precision == blp.BLP_FP64 else 1e-7
        assert rel(d[1][0], oracle.band_solve(N, A, f2)) <= tol


def test_default_is_the_host_loop(monkeypatch):
    N, eps = 64, 1e-4
    p, _ = problem(N, eps)
    monkeypatch.delenv("BLP_SOLVE_GRAPH", raising=False)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r))
    _, info = s.solve(T(p.f))
    s.close()
    assert info.status == 0 and info.device_driven == 0


def test_unscaled_rule_keeps_the_host_loop(monkeypatch):
    """The unscaled stopping rules convert their target between restarts on
    the host, so they keep the host-driven loop."""
    N, eps = 64, 1e-4
    p, _ = problem(N, eps)
    monkeypatch.delenv("BLP_SOLVE_GRAPH", raising=False)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), stop_mode=blp.BLP_STOP_REL2, device_driven=1)
    _, info = s.solve(T(p.f))
    s.close()
    assert info.status == 0 and info.device_driven == 0

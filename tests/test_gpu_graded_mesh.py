"""The solve on the graded (Bakhvalov-Shishkin) layer mesh through the C ABI
(BLP_MESH_GRADED; the Remark after Theorem (big bound) covers graded layer
meshes).  Same blocks, kernels and tolerances as on the Shishkin mesh:
preconditioner against the oracle's (FP64 1e-11, same cycle counts; FP32
1e-4 at a fixed cycle count), solves against the oracle's direct solve
(FP64 1e-8, mixed 1e-7), and at N = 512 / 1024, beyond the direct solver's
reach, the convergence property the mesh is built for: first order in N
without the ln N factor, below the Shishkin error."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2108_13468_gb300 as blp  # noqa: E402
from paper_2108_13468_gb300 import inputs  # noqa: E402


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    a = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def problem(N, eps, seed=0):
    x, _ = oracle.mesh(N, eps, graded=True)
    p = inputs.problem_fourier_quadratic(x, x, N, eps, seed=seed)
    return x, p, oracle.assemble(N, eps, x, x, p.c1, p.c2, p.r)


@pytest.mark.parametrize("N,eps", [(96, 1e-4), (130, 1e-8), (130, 1e-2)])
def test_graded_preconditioner_matches_oracle(N, eps):
    x, p, A = problem(N, eps)
    v = np.random.default_rng(3).standard_normal((N - 1) ** 2)
    P = oracle.Prec(N, eps, x, x, p.c1, p.c2, p.r)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), mesh=blp.BLP_MESH_GRADED)
    zo, co = P.apply(A["C"] * v)
    z, c = s.precond(T(v))
    assert c == co and rel(z, zo) < 1e-11
    zto, cto = P.apply(v, transpose=True)
    zt, ct = s.precond(T(v), transpose=True)
    assert ct == cto and rel(zt, A["C"] * zto) < 1e-11
    P3 = oracle.Prec(N, eps, x, x, p.c1, p.c2, p.r, fixed_cycles=3)
    s3 = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), mesh=blp.BLP_MESH_GRADED, corner_fixed_cycles=3)
    assert rel(s3.precond(T(v), precision=blp.BLP_MIXED)[0], P3.apply(A["C"] * v)[0]) < 1e-4


@pytest.mark.parametrize("N,eps", [(64, 1e-2), (128, 1e-6), (256, 1e-4)])
@pytest.mark.parametrize("precision,tol", [(blp.BLP_FP64, 1e-8), (blp.BLP_MIXED, 1e-7)])
def test_graded_solve_matches_direct(N, eps, precision, tol):
    x, p, A = problem(N, eps, seed=1)
    ue = oracle.band_solve(N, A, p.f)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), precision=precision, mesh=blp.BLP_MESH_GRADED)
    u, info = s.solve(T(p.f), tol=1e-10)
    assert info.status == 0 and rel(u, ue) <= tol


def mms_error(N, eps, mesh):
    graded = mesh == blp.BLP_MESH_GRADED
    x, _ = blp.mesh(N, eps, 2.5, 2.0, graded=graded)
    y, _ = blp.mesh(N, eps, 2.5, 3.0, graded=graded)
    f, ue = inputs.mms_exponential(x, y, eps)
    one = np.ones_like(f)
    s = blp.Solver(N, eps, T(2.0 * one), T(3.0 * one), T(one), sigma=2.5, beta_x=2.0, beta_y=3.0, mesh=mesh)
    u, info = s.solve(T(f), tol=1e-12)
    s.close()
    assert info.status == 0
    return float(np.abs(u.cpu().numpy() - ue).max())


def test_graded_mesh_first_order_at_large_n():
    eps = 1e-6
    eg = [mms_error(N, eps, blp.BLP_MESH_GRADED) for N in (512, 1024)]
    es = [mms_error(N, eps, blp.BLP_MESH_SHISHKIN) for N in (512, 1024)]
    rate_g, rate_s = np.log2(eg[0] / eg[1]), np.log2(es[0] / es[1])
    assert eg[0] < es[0] and eg[1] < es[1]
    assert 0.97 <= rate_g <= 1.02                                   # N^-1, no ln N
    assert rate_s <= np.log2(2 * np.log(512) / np.log(1024)) + 0.02   # N^-1 ln N

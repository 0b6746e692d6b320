"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 path relative max-norm error <= 1e-8 against the oracle's
direct solve (the target stated for the method), mixed path <= 1e-7; the
FP64 preconditioner and operator agree to rounding (1e-11); the FP32
preconditioner to 1e-4 (single precision through a few thousand sweeps of
a triangular recurrence with |couplings| <= 1)."""
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
    x, _ = oracle.mesh(N, eps)
    p = inputs.problem_fourier_quadratic(x, x, N, eps, seed=seed)
    return x, p, oracle.assemble(N, eps, x, x, p.c1, p.c2, p.r)


CASES = [(8, 1e-3), (10, 1e-6), (66, 1e-2), (66, 1e-8), (96, 1e-4), (128, 1e-4), (128, 1e-8)]


@pytest.mark.parametrize("N,eps", CASES)
def test_operator_apply(N, eps):
    x, p, A = problem(N, eps)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r))
    v = np.random.default_rng(1).standard_normal((N - 1) ** 2)
    assert rel(s.apply(T(v)), oracle.apply(N, A, v)) < 1e-13
    assert rel(s.apply(T(v), transpose=True), oracle.apply(N, A, v, transpose=True)) < 1e-13


@pytest.mark.parametrize("N,eps", CASES)
@pytest.mark.parametrize("fixed", [0, 3])
def test_preconditioner(N, eps, fixed):
    """z = (D^-1 M)^-1 v = M^-1 (D v) and z = (D^-1 M)^-T v = D M^-T v."""
    x, p, A = problem(N, eps)
    P = oracle.Prec(N, eps, x, x, p.c1, p.c2, p.r, fixed_cycles=fixed)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), corner_fixed_cycles=fixed)
    v = np.random.default_rng(2).standard_normal((N - 1) ** 2)
    zo, co = P.apply(A["C"] * v)
    z, c = s.precond(T(v))
    assert c == co and rel(z, zo) < 1e-11
    zto, cto = P.apply(v, transpose=True)
    zt, ct = s.precond(T(v), transpose=True)
    assert ct == cto and rel(zt, A["C"] * zto) < 1e-11
    if fixed:   # FP32: same cycle count by construction
        assert rel(s.precond(T(v), precision=blp.BLP_MIXED)[0], zo) < 1e-4
        assert rel(s.precond(T(v), transpose=True, precision=blp.BLP_MIXED)[0], A["C"] * zto) < 1e-4


@pytest.mark.parametrize("N,eps", CASES)
@pytest.mark.parametrize("precision,tol", [(blp.BLP_FP64, 1e-8), (blp.BLP_MIXED, 1e-7)])
def test_solve_matches_direct(N, eps, precision, tol):
    x, p, A = problem(N, eps)
    ue = oracle.band_solve(N, A, p.f)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), precision=precision)
    u, info = s.solve(T(p.f), tol=1e-10)
    assert info.status == 0 and info.relres <= 1e-10
    assert rel(u, ue) <= tol
    # the oracle's own residual of the GPU answer (row-normalised system)
    un = u.cpu().numpy()
    r = (p.f - oracle.apply(N, A, un)) / A["C"]
    assert np.linalg.norm(r) <= 1.0001e-10 * np.linalg.norm(p.f / A["C"])


@pytest.mark.parametrize("N,eps", [(66, 1e-2), (128, 1e-4), (96, 1e-8)])
@pytest.mark.parametrize("precision", [blp.BLP_FP64, blp.BLP_MIXED])
def test_adjoint_and_gradient(N, eps, precision):
    x, p, A = problem(N, eps)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), precision=precision)
    g = np.random.default_rng(3).uniform(0, 1, (N - 1) ** 2)
    le = oracle.band_solve(N, A, g, transpose=True)
    lam, info = s.solve_adjoint(T(g), tol=1e-10)
    assert info.status == 0
    assert rel(lam, le) <= (1e-8 if precision == blp.BLP_FP64 else 1e-7)
    ue = oracle.band_solve(N, A, p.f)
    for a, b in zip(s.grad(T(ue), T(le)), oracle.grad(N, x, x, ue, le)):
        assert rel(a, b) < 1e-13


def test_host_pointers_match_device():
    N, eps = 96, 1e-4
    x, p, A = problem(N, eps)
    s = blp.Solver(N, eps, p.c1, p.c2, p.r)          # numpy (host) fields
    uh = np.zeros((N - 1) ** 2)
    _, info = s.solve(p.f.copy(), uh, tol=1e-10)
    ud, _ = s.solve(T(p.f), tol=1e-10)
    assert info.status == 0 and np.array_equal(uh, ud.cpu().numpy())


def test_edge_cases_and_errors():
    N, eps = 64, 1e-4
    x, p, A = problem(N, eps)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r))
    u, info = s.solve(T(np.zeros_like(p.f)))             # zero rhs: u = 0, no iterations
    assert info.status == 0 and info.iters == 0 and float(u.abs().max()) == 0.0
    ue = oracle.band_solve(N, A, p.f)
    u0 = T(ue + 1e-3 * np.sin(np.arange(ue.size)))         # good initial guess: few iterations
    u, info = s.solve(T(p.f), u0, tol=1e-10)
    assert info.status == 0 and rel(u, ue) < 1e-8
    s1 = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), maxit=1)
    u, info = s1.solve(T(p.f), tol=1e-14, raise_on_noconv=False)   # iteration cap: best iterate kept
    assert info.status == blp._native.BLP_ERR_NOCONV and info.iters == 1 and 0 < info.relres < 1
    with pytest.raises(blp.BlpError) as e:
        blp.Solver(N, eps, T(p.c1 - 0.5), T(p.c2), T(p.r))      # c1 below beta_x = 1
    assert e.value.status == blp._native.BLP_ERR_COEF
    bad = p.r.copy()
    bad[5] = np.nan
    with pytest.raises(blp.BlpError):
        blp.Solver(N, eps, T(p.c1), T(p.c2), T(bad))
    one = T(np.ones(62 * 62))
    with pytest.raises(blp.BlpError) as e:
        blp.Solver(63, eps, one, one, one)                         # odd N: rejected by blp_setup
    assert e.value.status == blp._native.BLP_ERR_ARG


@pytest.mark.parametrize("eps", [1e-4, 1e-8])
def test_full_size_n1024(eps):
    """N = 1024 (the benchmark workload): operator and FP64 preconditioner
    against the oracle on the whole vector, and both solves checked by the
    oracle's own residual (a property that holds at any size) plus the
    oracle's FGMRES answer at a tighter tolerance."""
    N = 1024
    x, p, A = problem(N, eps)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r))
    v = np.random.default_rng(4).standard_normal((N - 1) ** 2)
    assert rel(s.apply(T(v)), oracle.apply(N, A, v)) < 1e-13
    P = oracle.Prec(N, eps, x, x, p.c1, p.c2, p.r)
    zo, co = P.apply(A["C"] * v)
    z, c = s.precond(T(v))
    assert c == co and rel(z, zo) < 1e-10
    uo, st, it, rr, mc = oracle.fgmres(N, A, p.f, P, tol=1e-13)
    assert st == 0
    for prec, tol in ((blp.BLP_FP64, 1e-8), (blp.BLP_MIXED, 1e-7)):
        sp = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), precision=prec)
        u, info = sp.solve(T(p.f), tol=1e-10)
        un = u.cpu().numpy()
        r = (p.f - oracle.apply(N, A, un)) / A["C"]
        assert info.status == 0 and np.linalg.norm(r) <= 1.0001e-10 * np.linalg.norm(p.f / A["C"])
        assert rel(un, uo) <= tol


# (BLP_DTS_TWO_STEP, BLP_DTS_CHUNK, BLP_DTS_CLUSTER): both forms of the
# wavefront recurrence, every hand-off chunk, and cluster sizes that put the
# strips in one wave (8, 16) or in several waves handed over through global
# memory (1, 2)
WAVEFRONT_VARIANTS = [("0", "0", "8"), ("3", "0", "8"), ("3", "8", "8"), ("3", "16", "1"), ("3", "32", "1"),
                      ("0", "32", "2"), ("3", "16", "16")]


@pytest.mark.parametrize("N", [512, 514, 1024])
def test_wavefront_forms_and_shapes(N, monkeypatch):
    """The one- and two-step forms of the downstream sweep (Sec. 3.1, 3.2),
    under every chunk length and cluster shape, against the oracle's
    preconditioner. N = 512: interior 255^2 (ragged last strip), corner
    256^2 -> 128^2 -> 64^2 on the wavefront kernel; N = 514: corner 257^2 (a
    one-column last strip, a single level of 4 sweeps per cycle); N = 1024:
    16-strip blocks, which a one-CTA cluster (15 compute warps at most)
    processes in two waves. Fixed cycle count, so FP32 and FP64 apply the
    same operator. FP32 bound: one rounding (2^-24) per step along the ~2N
    dependent steps of a sweep, with a factor 4 for the cycles and levels:
    8 N 2^-24 (2.4e-4 at N = 512, 4.9e-4 at N = 1024)."""
    tol32 = 8 * N * 2.0 ** -24
    eps, fixed = 1e-4, 2
    x, p, A = problem(N, eps)
    P = oracle.Prec(N, eps, x, x, p.c1, p.c2, p.r, fixed_cycles=fixed)
    v = np.random.default_rng(6).standard_normal((N - 1) ** 2)
    zo, _ = P.apply(A["C"] * v)
    zto, _ = P.apply(v, transpose=True)
    zto = A["C"] * zto
    for two_step, chunk, cluster in WAVEFRONT_VARIANTS:
        monkeypatch.setenv("BLP_DTS_TWO_STEP", two_step)
        monkeypatch.setenv("BLP_DTS_CHUNK", chunk)
        monkeypatch.setenv("BLP_DTS_CLUSTER", cluster)
        s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), corner_fixed_cycles=fixed)
        tag = (two_step, chunk, cluster)
        assert rel(s.precond(T(v))[0], zo) < 1e-11, tag
        assert rel(s.precond(T(v), transpose=True)[0], zto) < 1e-11, tag
        assert rel(s.precond(T(v), precision=blp.BLP_MIXED)[0], zo) < tol32, tag
        assert rel(s.precond(T(v), transpose=True, precision=blp.BLP_MIXED)[0], zto) < tol32, tag
        s.close()

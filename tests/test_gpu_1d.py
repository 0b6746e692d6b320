"""The one-dimensional method of Sec. 2 on the GPU (blp_solve_1d_batched):
upwind scheme on the Shishkin mesh of eq. (tau 1D), GMRES without restarts on
the left-preconditioned system with M of eq. (block_M) (the setting of
Table 2), stopping on the true residual ||f - A u||_inf <= K g(N) (Sec. 2.5.1,
K = ||U^E||_inf, g(N) = ln(N)/N), on the problem of eq. (1D example).

Parity: every Table 2 count exactly, the oracle's GMRES count and its iterate
(left-preconditioned, `oracle.oned`), the returned residual against the
oracle's matrix, and the error bound
||u - U^E||_inf <= ||A^-1||_inf ||f - A u||_inf <= 2 stop (barrier W = 2 - x,
A W >= C_low).  The oracle side is built on the oracle's own mesh
(`oned.mesh`, C_low = 0.99, the constant that reproduces Table 1) and the GPU
receives the fields sampled at those nodes, so a mesh error in the library
shows up as a mismatch.  The unscaled residual has a rounding floor: entries
of A that differ by rounding move f - A u by up to a few ulps of |A| |u|
(16 ulps here, floor = 16 2^-53 || |A| |u| ||_inf, 1e-3 at N = 1024,
eps = 1e-8), and the oracle applies M^-1 through a dense inverse, so iterates
and residuals are compared to 1e-9 relative plus twice that floor.  Also: a
tight stop against the direct solve, one thread per problem (a problem's
answer does not depend on the batch around it), and the argument checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_13468_gb300 as blp  # noqa: E402
from oracle import oned  # noqa: E402
from paper_2108_13468_gb300 import _native  # noqa: E402
from tests.conftest import read_table  # noqa: E402

c = lambda x: 2.0 + np.sin(5.0 * x)        # noqa: E731  eq. (1D example)
r = lambda x: 1.0 + 0.0 * x                # noqa: E731
f = lambda x: 4.0 * np.exp(-x)             # noqa: E731


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


C_LOW = 0.99   # the transition-point constant that reproduces Table 1 (eq. tau 1D)


def gpu_problem(N, eps, stop, maxit=64):
    x, _, _ = oned.mesh(N, eps, C_LOW)         # fields sampled at the oracle's nodes
    xi = x[1:-1]
    return dict(N=N, eps=eps, c=T(c(xi)), r=T(r(xi)), f=T(f(xi)), stop=stop, maxit=maxit, c_low=C_LOW)


def oracle_problem(N, eps):
    x, _, NL = oned.mesh(N, eps, C_LOW)
    A = oned.dense(*oned.assemble(x, eps, c, r))
    b = f(x[1:-1])
    return A, b, NL, np.linalg.solve(A, b)


def floor(A, u):
    return 16 * 2.0 ** -53 * np.abs(np.abs(A) @ np.abs(u)).max()


def test_table2_iteration_counts_batched():
    header, rows = read_table("table2_1d_iterations.txt")
    Ns = [int(h.split("=")[1]) for h in header]
    cases = [(float(e), N, int(ref)) for e, vals in rows.items() for N, ref in zip(Ns, vals) if ref is not None]
    probs, orc = [], []
    for eps, N, ref in cases:
        A, b, NL, UE = oracle_problem(N, eps)
        stop = np.abs(UE).max() * np.log(N) / N
        probs.append(gpu_problem(N, eps, stop))
        orc.append((A, b, NL, UE, stop))
    res = blp.solve_1d_batched(probs)                      # every Table 2 problem in one launch
    for (eps, N, ref), (A, b, NL, UE, stop), (u, it, resid, st) in zip(cases, orc, res):
        un = u.cpu().numpy()
        fl = floor(A, un)
        assert st == _native.BLP_OK and it == ref, (eps, N, it, ref)
        ores = np.abs(b - A @ un).max()
        assert ores <= stop + fl and abs(resid - ores) <= fl, (eps, N, resid, ores, fl)
        assert np.abs(un - UE).max() <= 2.0 * (stop + fl)
        xo, ito = oned.gmres_left_true_residual(A, b, oned.block_M(A, NL), stop)
        assert it == ito, (eps, N, it, ito)
        assert np.abs(un - xo).max() <= 1e-9 * np.abs(xo).max() + 2 * fl, (eps, N)


def test_tight_stop_matches_direct_solve():
    N, eps = 64, 1e-2
    A, b, NL, UE = oracle_problem(N, eps)
    stop = 1e-10 * np.abs(b).max()           # above the residual's rounding floor (~1e-11 here)
    (u, it, resid, st), = blp.solve_1d_batched([gpu_problem(N, eps, stop, maxit=64)])
    assert st == _native.BLP_OK and resid <= stop
    assert np.abs(u.cpu().numpy() - UE).max() <= 2.0 * (stop + floor(A, u.cpu().numpy()))   # ~1e-10 relative


def test_one_thread_per_problem_is_independent_of_the_batch():
    specs = [(8, 1e-3), (10, 1e-6), (130, 1e-4), (4096, 1e-8), (2048, 1e-5), (8, 1e-3)]
    probs = [gpu_problem(N, eps, 4.0 * np.log(N) / N) for N, eps in specs]
    res = blp.solve_1d_batched(probs)
    for p, (u, it, resid, st) in zip(probs, res):
        (u1, it1, resid1, st1), = blp.solve_1d_batched([p])
        assert st == st1 == _native.BLP_OK and it == it1 and resid == resid1
        assert torch.equal(u, u1)


def test_argument_checks_and_iteration_cap():
    good = gpu_problem(64, 1e-4, 1e-3)
    odd = dict(good, N=63, **{k: good[k][:62].contiguous() for k in ("c", "r", "f")})
    with pytest.raises(blp.BlpError) as e:
        blp.solve_1d_batched([good, odd])                     # odd N: refused by the library, nothing runs
    assert e.value.status == _native.BLP_ERR_ARG
    x, _, _ = oned.mesh(64, 1e-4, C_LOW)
    host = dict(good, f=np.ascontiguousarray(f(x[1:-1])))  # a host array is refused, never dereferenced
    with pytest.raises(blp.BlpError):
        blp.solve_1d_batched([host])
    with pytest.raises(blp.BlpError):
        blp.solve_1d_batched([dict(good, maxit=_native.BLP_1D_MAXIT + 1)])
    (u, it, resid, st), = blp.solve_1d_batched([dict(good, stop=0.0, maxit=1)])   # unreachable: cap
    assert st == _native.BLP_ERR_NOCONV and it == 1 and resid > 0.0

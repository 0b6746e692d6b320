"""blp_residual_noalloc, the residual call that allocates nothing, against the
handle-based operator (blp_apply_operator) and the handle-based solve.

Two calls in a row with different sizes check that the shared fixed scratch
carries nothing from one call to the next.  Tolerance: the two paths evaluate
the same stencil in different association orders, so entries agree to
1e-13 of max |aC u| (a few ulps of the largest term of a row), and the norms
of a residual that is not itself rounding noise to 1e-12 relative."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2108_13468_gb300 as blp  # noqa: E402
from paper_2108_13468_gb300 import _native, inputs  # noqa: E402


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def P(t):
    return ctypes.c_void_p(t.data_ptr())


def case(N, eps, seed):
    x, _ = oracle.mesh(N, eps)
    p = inputs.problem_fourier_quadratic(x, x, N, eps, seed=seed)
    u = np.random.default_rng(seed + 10).standard_normal((N - 1) ** 2)
    return dict(N=N, eps=eps, x=x, p=p, u=u, dev=[T(a) for a in (x, x, p.c1, p.c2, p.r, p.f, u)])


def noalloc(lib, c, res):
    norms = np.full(4, np.nan)
    d = c["dev"]
    st = lib.blp_residual_noalloc(c["N"], P(d[0]), P(d[1]), c["eps"], *[P(t) for t in d[2:]], P(res),
                                  ctypes.c_void_p(norms.ctypes.data), ctypes.c_void_p(None))
    assert st == _native.BLP_OK, lib.blp_strerror(st)
    return norms


def reference(c):
    """f - A u through blp_apply_operator, and D from the oracle's assembly."""
    N, eps, p = c["N"], c["eps"], c["p"]
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r))
    Au = s.apply(T(c["u"])).cpu().numpy()
    s.close()
    D = oracle.assemble(N, eps, c["x"], c["x"], p.c1, p.c2, p.r)["C"]
    return p.f - Au, D, np.abs(D * c["u"]).max()


def test_noalloc_residual_matches_apply_operator_twice():
    lib = _native.load()
    cases = [case(128, 1e-4, 0), case(66, 1e-8, 1)]
    refs = [reference(c) for c in cases]
    outs = [torch.full(((c["N"] - 1) ** 2,), float("nan"), dtype=torch.float64, device="cuda") for c in cases]
    norms = [noalloc(lib, c, o) for c, o in zip(cases, outs)]   # two calls in a row
    for c, (s_ref, D, scale), o, nr in zip(cases, refs, outs, norms):
        s = o.cpu().numpy()
        f = c["p"].f
        assert np.abs(s - s_ref).max() <= 1e-13 * scale
        want = [np.linalg.norm(s_ref), np.linalg.norm(s_ref / D), np.linalg.norm(f), np.linalg.norm(f / D)]
        np.testing.assert_allclose(nr, want, rtol=1e-12)


def test_noalloc_norms_of_a_solution_match_blp_solve():
    lib = _native.load()
    c = case(96, 1e-6, 2)
    p = c["p"]
    s = blp.Solver(c["N"], c["eps"], T(p.c1), T(p.c2), T(p.r))
    u, info = s.solve(T(p.f), tol=1e-10)
    s.close()
    c["dev"][6] = u
    out = torch.empty_like(u)
    for _ in range(2):
        nr = noalloc(lib, c, out)
        assert abs(nr[1] / nr[3] - info.relres) <= 0.05 * info.relres
        assert abs(nr[0] / nr[2] - info.relres_unscaled) <= 0.05 * info.relres_unscaled


def test_noalloc_rejects_sizes_beyond_its_limit_and_host_arrays():
    lib = _native.load()
    c = case(8, 1e-2, 3)
    d = c["dev"]
    args = [P(t) for t in d[2:]]
    big = _native.BLP_NOALLOC_MAX_N + 2
    # rejected on the host before any device work (the small buffers are never read)
    assert lib.blp_residual_noalloc(big, P(d[0]), P(d[1]), 1e-2, *args, None, None, None) == _native.BLP_ERR_ARG
    assert lib.blp_residual_noalloc(9, P(d[0]), P(d[1]), 1e-2, *args, None, None, None) == _native.BLP_ERR_ARG
    host_x = np.ascontiguousarray(c["x"])
    assert lib.blp_residual_noalloc(8, ctypes.c_void_p(host_x.ctypes.data), P(d[1]), 1e-2, *args, None, None,
                                    None) == _native.BLP_ERR_ARG
    with pytest.raises(ValueError, match="no-allocation limit"):
        blp.residual_noalloc(big, *d[:2], 1e-2, *d[2:])
    # the binding returns the same norms as the raw call
    np.testing.assert_array_equal(blp.residual_noalloc(8, *d[:2], 1e-2, *d[2:]),
                                  noalloc(lib, c, torch.empty_like(d[6])))

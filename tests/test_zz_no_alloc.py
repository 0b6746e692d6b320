"""blp_residual_noalloc, the residual call that allocates nothing, against the
oracle's assembly and operator apply.

It serves callers that cannot allocate device memory when they check a
solution (memory already fully reserved, or a path where cudaMalloc's
device-wide synchronisation would stall other streams).  Two calls in a row
with different sizes check that the shared fixed scratch carries nothing from
one call to the next.  Tolerance: the two sides evaluate the same stencil in
different association orders, so entries agree to 1e-13 of max |aC u| (a few
ulps of the largest term of a row), and the norms of a residual that is not
itself rounding noise to 1e-12 relative."""
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


def reference(c, u=None):
    """s = f - A u and D = diag(A) from the oracle's own assembly and apply."""
    N, eps, p = c["N"], c["eps"], c["p"]
    u = c["u"] if u is None else u
    A = oracle.assemble(N, eps, c["x"], c["x"], p.c1, p.c2, p.r)
    s = p.f - oracle.apply(N, A, u)
    return s, A["C"], np.abs(A["C"] * u).max()


def want_norms(s, D, f):
    return [np.linalg.norm(s), np.linalg.norm(s / D), np.linalg.norm(f), np.linalg.norm(f / D)]


def test_noalloc_residual_matches_the_oracle_twice():
    lib = _native.load()
    cases = [case(128, 1e-4, 0), case(66, 1e-8, 1)]
    refs = [reference(c) for c in cases]
    outs = [torch.full(((c["N"] - 1) ** 2,), float("nan"), dtype=torch.float64, device="cuda") for c in cases]
    norms = [noalloc(lib, c, o) for c, o in zip(cases, outs)]   # two calls in a row
    for c, (s_ref, D, scale), o, nr in zip(cases, refs, outs, norms):
        s = o.cpu().numpy()
        assert np.abs(s - s_ref).max() <= 1e-13 * scale
        np.testing.assert_allclose(nr, want_norms(s_ref, D, c["p"].f), rtol=1e-12)


def test_noalloc_without_res_and_with_device_norms():
    """res = NULL still gives the four norms; norms may live on the device."""
    lib = _native.load()
    c = case(96, 1e-6, 4)
    s_ref, D, _ = reference(c)
    want = want_norms(s_ref, D, c["p"].f)
    d = c["dev"]
    host = np.full(4, np.nan)
    st = lib.blp_residual_noalloc(c["N"], P(d[0]), P(d[1]), c["eps"], *[P(t) for t in d[2:]], None,
                                  ctypes.c_void_p(host.ctypes.data), None)
    assert st == _native.BLP_OK
    np.testing.assert_allclose(host, want, rtol=1e-12)
    dev = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.blp_residual_noalloc(c["N"], P(d[0]), P(d[1]), c["eps"], *[P(t) for t in d[2:]], None, P(dev), None)
    assert st == _native.BLP_OK
    np.testing.assert_allclose(dev.cpu().numpy(), want, rtol=1e-12)


def test_noalloc_norms_of_a_solution_match_the_oracle():
    """The norms of a computed solution, against the oracle's residual of the
    same u, on two calls in a row; the solve met its tolerance by them."""
    lib = _native.load()
    c = case(96, 1e-6, 2)
    p = c["p"]
    s = blp.Solver(c["N"], c["eps"], T(p.c1), T(p.c2), T(p.r))
    u, info = s.solve(T(p.f), tol=1e-10)
    s.close()
    c["dev"][6] = u
    s_ref, D, _ = reference(c, u.cpu().numpy())
    want = want_norms(s_ref, D, p.f)
    out = torch.empty_like(u)
    for _ in range(2):
        nr = noalloc(lib, c, out)
        # a converged residual is itself rounding-sized: compare to the oracle
        # to a few ulps of |A| |u| summed in quadrature over the grid
        fl = 16 * 2.0 ** -53 * np.linalg.norm(np.abs(D * u.cpu().numpy())) * 4
        assert abs(nr[0] - want[0]) <= fl and abs(nr[1] - want[1]) <= fl / D.min()
        np.testing.assert_allclose(nr[2:], want[2:], rtol=1e-12)
        assert nr[1] / nr[3] <= 1.05e-10


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
    pinned = torch.from_numpy(host_x).pin_memory()          # page-locked host memory is refused too
    assert lib.blp_residual_noalloc(8, P(pinned), P(d[1]), 1e-2, *args, None, None, None) == _native.BLP_ERR_ARG
    with pytest.raises(ValueError, match="no-allocation limit"):
        blp.residual_noalloc(big, *d[:2], 1e-2, *d[2:])
    # the binding returns the same norms as the raw call
    np.testing.assert_array_equal(blp.residual_noalloc(8, *d[:2], 1e-2, *d[2:]),
                                  noalloc(lib, c, torch.empty_like(d[6])))

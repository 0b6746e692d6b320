"""The closed-form forcings of the manufactured problems (Sec. 3.3, eqs.
exponential_MMS and parabolic_MMS) in inputs.py equal the symbolic ones
(sympy), so the GPU tests that reproduce the paper's tables start from the
paper's problems."""
import numpy as np
import pytest

import oracle
from paper_2108_13468_gb300 import inputs


def test_exponential_mms_forcing_matches_symbolic():
    sp = pytest.importorskip("sympy")
    X, Y, E = sp.symbols("x y eps", positive=True)
    u = sp.cos(sp.pi * X / 2) * (1 - sp.exp(-2 * X / E)) * (1 - Y) ** 3 * (1 - sp.exp(-3 * Y / E))
    f = -E * (sp.diff(u, X, 2) + sp.diff(u, Y, 2)) - 2 * sp.diff(u, X) - 3 * sp.diff(u, Y) + u
    uf, ff = sp.lambdify((X, Y, E), u, "numpy"), sp.lambdify((X, Y, E), f, "numpy")
    for N, eps in ((32, 1e-2), (64, 1e-4), (128, 1e-7)):
        x, _ = oracle.mesh(N, eps, 2.5, 2.0)
        y, _ = oracle.mesh(N, eps, 2.5, 3.0)
        f_, u_ = inputs.mms_exponential(x, y, eps)
        XX, YY = inputs.interior_grid(x, y)
        with np.errstate(all="ignore"):
            fs, us = ff(XX, YY, eps), uf(XX, YY, eps)
        np.testing.assert_allclose(u_, us, rtol=1e-12, atol=1e-14)
        # f is a difference of terms of size ~4/eps near the layers: rounding of
        # the two evaluation orders scales with 1/eps; a wrong or dropped term
        # would differ by O(1) relative
        np.testing.assert_allclose(f_, fs, rtol=1e-9, atol=1e-14 / eps)


def test_parabolic_mms_forcing_matches_symbolic():
    sp = pytest.importorskip("sympy")
    X, Y, E = sp.symbols("x y eps", positive=True)
    u = (sp.cos(sp.pi * X / 2) - (sp.exp(-X / E) - sp.exp(-1 / E)) / (1 - sp.exp(-1 / E))) * \
        ((1 - sp.exp(-Y / sp.sqrt(E))) / (1 - sp.exp(-1 / sp.sqrt(E))) - Y ** sp.Rational(5, 2))
    f = -E * (sp.diff(u, X, 2) + sp.diff(u, Y, 2)) - sp.diff(u, X) + u
    uf, ff = sp.lambdify((X, Y, E), u, "numpy"), sp.lambdify((X, Y, E), f, "numpy")
    for N, eps in ((32, 1e-2), (64, 1e-4), (128, 1e-7)):
        x, _ = oracle.mesh(N, eps, 2.5, 1.0)
        y, _ = oracle.mesh(N, eps, 2.5, 1.0, parabolic=True)
        f_, u_ = inputs.mms_parabolic(x, y, eps)
        XX, YY = inputs.interior_grid(x, y)
        with np.errstate(all="ignore"):
            fs, us = ff(XX, YY, eps), uf(XX, YY, eps)
        np.testing.assert_allclose(u_, us, rtol=1e-12, atol=1e-14)
        # the symbolic form subtracts two terms of size ~1/eps near x = 0 that
        # the closed form cancels exactly: its rounding scales with 1/eps
        np.testing.assert_allclose(f_, fs, rtol=1e-9, atol=1e-14 / eps)

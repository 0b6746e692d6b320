"""FP64 CPU oracle for the boundary-layer preconditioned solve (arXiv 2108.13468).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The product library
never imports, links or calls anything here, and nothing here imports the
product library.

The arithmetic lives in ``blp_oracle.c`` (plain sequential C, double
precision).  This module only marshals numpy arrays into it.  Interior
vectors are (N-1)**2 long, x-fastest: k = (j-1)*(N-1) + (i-1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "blp_oracle.c")
_LIB = os.path.join(_HERE, "libblp_oracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    c_int, c_double, c_void = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    lib.orc_mesh.restype = c_double
    lib.orc_mesh.argtypes = [c_int, c_double, c_double, c_double, c_int, _D]
    lib.orc_assemble_grid.restype = None
    lib.orc_assemble_grid.argtypes = [c_int, c_int, _D, _D, c_double, _D, _D, _D, _D, _D, _D, _D, _D]
    lib.orc_apply.restype = None
    lib.orc_apply.argtypes = [c_int, _D, _D, _D, _D, _D, _D, _D, c_int]
    lib.orc_band_solve.restype = c_int
    lib.orc_band_solve.argtypes = [c_int, _D, _D, _D, _D, _D, _D, _D, c_int]
    lib.orc_prec_create.restype = c_void
    lib.orc_prec_create.argtypes = [c_int, c_double, _D, _D, _D, _D, _D, c_double, c_int, c_int, c_int, c_int, c_int]
    lib.orc_prec_create_split.restype = c_void
    lib.orc_prec_create_split.argtypes = [c_int, c_int, c_double, _D, _D, _D, _D, _D, c_double, c_int, c_int, c_int,
                                          c_int, c_int]
    lib.orc_prec_set_distance.restype = None
    lib.orc_prec_set_distance.argtypes = [c_void, c_int]
    lib.orc_mesh_q.restype = c_double
    lib.orc_mesh_q.argtypes = [c_int, c_int, c_double, c_double, c_double, _D]
    lib.orc_semi_nlev.restype = c_int
    lib.orc_semi_nlev.argtypes = [c_void]
    lib.orc_semi_width.restype = c_int
    lib.orc_semi_width.argtypes = [c_void, c_int]
    lib.orc_semi_level.restype = None
    lib.orc_semi_level.argtypes = [c_void, c_int, _D, _D, _D]
    lib.orc_semi_gs.restype = None
    lib.orc_semi_gs.argtypes = [c_void, c_int, _D, _D]
    lib.orc_prec_destroy.restype = None
    lib.orc_prec_destroy.argtypes = [c_void]
    lib.orc_prec_apply.restype = c_int
    lib.orc_prec_apply.argtypes = [c_void, _D, _D, c_int]
    lib.orc_prec_nlev.restype = c_int
    lib.orc_prec_nlev.argtypes = [c_void]
    lib.orc_prec_level_size.restype = c_int
    lib.orc_prec_level_size.argtypes = [c_void, c_int]
    lib.orc_prec_level.restype = None
    lib.orc_prec_level.argtypes = [c_void, c_int, _D, _D, _D, _D, _D, _D, _D, _D]
    lib.orc_mg_gs.restype = None
    lib.orc_mg_gs.argtypes = [c_void, c_int, _D, _D, c_int]
    lib.orc_mg_vcycle.restype = None
    lib.orc_mg_vcycle.argtypes = [c_void, c_int, _D, _D, c_int]
    lib.orc_mg_prolong.restype = None
    lib.orc_mg_prolong.argtypes = [c_void, c_int, _D, _D]
    lib.orc_mg_restrict.restype = None
    lib.orc_mg_restrict.argtypes = [c_void, c_int, _D, _D, c_int]
    lib.orc_corner_solve.restype = c_int
    lib.orc_corner_solve.argtypes = [c_void, _D, _D, c_int]
    lib.orc_fgmres.restype = c_int
    lib.orc_fgmres.argtypes = [c_void, c_int, _D, _D, _D, _D, _D, _D, _D, c_double, c_int, c_int, c_int,
                               c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_double), ctypes.POINTER(c_int)]
    lib.orc_grad.restype = None
    lib.orc_grad.argtypes = [c_int, _D, _D, _D, _D, _D, _D, _D]
    _lib = lib
    return lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


COEFS = ("W", "E", "S", "N", "C")


def mesh(N: int, eps: float, sigma: float = 2.0, beta: float = 1.0, parabolic: bool = False, graded: bool = False,
         layer_intervals: int | None = None):
    """Shishkin mesh nodes x[0..N] and the transition point tau (Sec. 2.2, Sec. 3).

    graded=True: the graded (Bakhvalov-Shishkin) layer mesh with the same tau
    and N/2 split (the Remark after Theorem (big bound) covers graded meshes).
    layer_intervals=NL: the general Shishkin mesh of the Remark on general
    Shishkin meshes, NL = qN intervals on [0, tau], tau = min(q, ...)."""
    assert not (parabolic and graded)
    x = np.zeros(N + 1)
    if layer_intervals is not None:
        assert not (parabolic or graded)
        tau = _load().orc_mesh_q(N, int(layer_intervals), eps, sigma, beta, _p(x))
        return x, tau
    tau = _load().orc_mesh(N, eps, sigma, beta, 1 if parabolic else (2 if graded else 0), _p(x))
    return x, tau


def assemble_grid(mx, my, xs, ys, eps, c1, c2, r):
    """Upwind 5-point stencil on an mx-by-my node block (Sec. 3)."""
    out = [np.zeros(mx * my) for _ in range(5)]
    _load().orc_assemble_grid(mx, my, _p(_f64(xs)), _p(_f64(ys)), eps, _p(_f64(c1)), _p(_f64(c2)),
                              _p(_f64(r)), *[_p(o) for o in out])
    return dict(zip(COEFS, out))


def assemble(N, eps, x, y, c1, c2, r):
    return assemble_grid(N - 1, N - 1, x, y, eps, c1, c2, r)


def apply(N, A, u, transpose=False):
    y = np.zeros((N - 1) ** 2)
    _load().orc_apply(N, *[_p(A[c]) for c in COEFS], _p(_f64(u)), _p(y), int(transpose))
    return y


def band_solve(N, A, f, transpose=False):
    """Direct solve by banded LU without pivoting (the oracle's exact answer)."""
    u = np.zeros((N - 1) ** 2)
    rc = _load().orc_band_solve(N, *[_p(A[c]) for c in COEFS], _p(_f64(f)), _p(u), int(transpose))
    if rc != 0:
        raise RuntimeError(f"orc_band_solve failed ({rc})")
    return u


def grad(N, x, y, u, lam):
    """(g_c1, g_c2, g_r) = -lam^T dA/dtheta u for the adjoint gradient."""
    g1, g2, gr = (np.zeros((N - 1) ** 2) for _ in range(3))
    _load().orc_grad(N, _p(_f64(x)), _p(_f64(y)), _p(_f64(u)), _p(_f64(lam)), _p(g1), _p(g2), _p(gr))
    return g1, g2, gr


class Prec:
    """The block preconditioner M of Sec. 3.1 (eq. 2D blocks) with the corner
    multigrid of Sec. 3.2.  fixed_cycles > 0 makes M_CC^{-1} a fixed number of
    cycles; corner_exact=True replaces M_CC by A_CC (the idealised M-hat).
    parabolic=True takes the corner cycle the paper gives for one parabolic
    and one exponential layer (x-semicoarsening, operator-induced
    interpolation, Galerkin coarse operators; forward application only); the
    paper stops it at a 10^2 reduction (pass reduction=1e2).
    layer_intervals=NL splits the blocks at layer index NL instead of N/2
    (the general Shishkin mesh of the Remark on general Shishkin meshes).
    distance_transfer=True interpolates linearly in the level coordinates
    (bilinear on a graded mesh) instead of with the index weights 1/2, 1/4."""

    def __init__(self, N, eps, x, y, c1, c2, r, reduction=1e3, max_cycles=50, fixed_cycles=0,
                 coarsest_min=2, corner_exact=False, parabolic=False, layer_intervals=None,
                 distance_transfer=False):
        self._lib = _load()
        self.N = N
        self.parabolic = parabolic
        self._keep = [_f64(a) for a in (x, y, c1, c2, r)]
        NL = N // 2 if layer_intervals is None else int(layer_intervals)
        h = self._lib.orc_prec_create_split(N, NL, eps, *[_p(a) for a in self._keep], reduction, max_cycles,
                                            fixed_cycles, coarsest_min, int(corner_exact), int(parabolic))
        if not h:
            raise ValueError("orc_prec_create rejected the arguments")
        self.h = ctypes.c_void_p(h)
        if distance_transfer:
            self._lib.orc_prec_set_distance(self.h, 1)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._lib.orc_prec_destroy(h)
            self.h = None

    def apply(self, v, transpose=False):
        if transpose and self.parabolic:
            raise ValueError("the parabolic corner cycle is provided forward only")
        z = np.zeros((self.N - 1) ** 2)
        cyc = self._lib.orc_prec_apply(self.h, _p(_f64(v)), _p(z), int(transpose))
        return z, cyc

    @property
    def nlev(self):
        return self._lib.orc_prec_nlev(self.h)

    def level_size(self, l):
        return self._lib.orc_prec_level_size(self.h, l)

    def level(self, l):
        m = self.level_size(l)
        xs, ys = np.zeros(m + 2), np.zeros(m + 2)
        arrs = [np.zeros(m * m) for _ in range(6)]
        self._lib.orc_prec_level(self.h, l, _p(xs), _p(ys), *[_p(a) for a in arrs])
        return xs, ys, dict(zip(COEFS + ("D",), arrs))

    @property
    def semi_nlev(self):
        return self._lib.orc_semi_nlev(self.h)

    def semi_level(self, l):
        """Level l of the parabolic cycle: (A9, PW, PE) with A9[(dy+1)*3+(dx+1)]
        the (m, width) array of entries to node (I+dx, J+dy), and the
        interpolation weights of the odd columns from level l+1."""
        w, m = self._lib.orc_semi_width(self.h, l), self.N // 2
        A9, PW, PE = np.zeros(9 * w * m), np.zeros(w * m), np.zeros(w * m)
        self._lib.orc_semi_level(self.h, l, _p(A9), _p(PW), _p(PE))
        return A9.reshape(9, m, w), PW.reshape(m, w), PE.reshape(m, w)

    def semi_gs(self, l, b, e):
        e = _f64(e).copy()
        self._lib.orc_semi_gs(self.h, l, _p(_f64(b)), _p(e))
        return e

    def gs(self, l, b, e, transpose=False):
        e = _f64(e).copy()
        self._lib.orc_mg_gs(self.h, l, _p(_f64(b)), _p(e), int(transpose))
        return e

    def vcycle(self, l, b, e, transpose=False):
        e = _f64(e).copy()
        self._lib.orc_mg_vcycle(self.h, l, _p(_f64(b)), _p(e), int(transpose))
        return e

    def prolong(self, l, ec):
        m = self.level_size(l)
        ef = np.zeros(m * m)
        self._lib.orc_mg_prolong(self.h, l, _p(_f64(ec)), _p(ef))
        return ef

    def restrict(self, l, rf, transpose=False):
        m = self.level_size(l + 1)
        bc = np.zeros(m * m)
        self._lib.orc_mg_restrict(self.h, l, _p(_f64(rf)), _p(bc), int(transpose))
        return bc

    def corner_solve(self, b, transpose=False):
        m = self.level_size(0)
        e = np.zeros(m * m)
        cyc = self._lib.orc_corner_solve(self.h, _p(_f64(b)), _p(e), int(transpose))
        return e, cyc


def fgmres(N, A, f, prec: Prec | None = None, tol=1e-10, tol_abs=False, restart=30, maxit=10000,
           transpose=False, u0=None, scaled=True):
    """Restarted FGMRES(restart) with MGS Arnoldi (Sec. 3.3).  scaled=True
    measures (and minimises) the residual of the row-normalised system
    diag(A)^{-1} A u = diag(A)^{-1} f.  Returns
    (u, status, iterations, relres, max_corner_cycles)."""
    u = np.zeros((N - 1) ** 2) if u0 is None else _f64(u0).copy()
    it, rr, mc = ctypes.c_int(0), ctypes.c_double(0.0), ctypes.c_int(0)
    st = _load().orc_fgmres(prec.h if prec is not None else None, N, *[_p(A[c]) for c in COEFS],
                            _p(_f64(f)), _p(u), tol, int(tol_abs), restart, maxit, int(transpose), int(scaled),
                            ctypes.byref(it), ctypes.byref(rr), ctypes.byref(mc))
    return u, st, it.value, rr.value, mc.value


def dense(N, A, transpose=False):
    """Dense copy of the assembled matrix (layout conversion only; tiny N)."""
    M = N - 1
    n = M * M
    D = np.zeros((n, n))
    for j in range(1, M + 1):
        for i in range(1, M + 1):
            p = (j - 1) * M + (i - 1)
            D[p, p] = A["C"][p]
            if i > 1:
                D[p, p - 1] = A["W"][p]
            if i < M:
                D[p, p + 1] = A["E"][p]
            if j > 1:
                D[p, p - M] = A["S"][p]
            if j < M:
                D[p, p + M] = A["N"][p]
    return D.T.copy() if transpose else D

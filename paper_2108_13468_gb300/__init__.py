"""GB300-native boundary-layer-preconditioned solver for singularly perturbed
convection-diffusion (MacLachlan, Madden & Nhan, arXiv 2108.13468).

Python surface over the C ABI of ``include/blp.h`` (libblp.so):

    x = mesh(N, eps)                       # Shishkin nodes (Sec. 3)
    s = Solver(N, eps, c1, c2, r)          # blp_setup: assembly + preconditioner
    u, info = s.solve(f, tol=1e-10)        # blp_solve: FGMRES + boundary-layer preconditioner
    lam, info = s.solve_adjoint(g)         # blp_solve_adjoint
    g1, g2, gr = s.grad(u, lam)            # blp_grad
    u = solve(f, c1, c2, r, N=..., eps=...)  # differentiable (torch.autograd.Function)

Arrays are float64 torch tensors (CUDA or CPU) or numpy arrays with
(N-1)**2 entries, x-fastest over the interior nodes.  All arithmetic runs in
libblp.so; this module only passes pointers.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N_
from ._native import (BLP_FP64, BLP_MESH_GRADED, BLP_MESH_PARABOLIC, BLP_MESH_SHISHKIN, BLP_MIXED, BLP_STOP_ABS2,
                      BLP_STOP_REL2, BLP_STOP_SCALED, BlpError, Info, Params)

__all__ = ["mesh", "Solver", "Params", "Info", "BlpError", "BLP_FP64", "BLP_MIXED", "BLP_STOP_SCALED",
           "BLP_STOP_REL2", "BLP_STOP_ABS2", "BLP_MESH_SHISHKIN", "BLP_MESH_GRADED", "BLP_MESH_PARABOLIC", "default_params",
           "solve",
           "solve_batched", "solve_1d_batched", "residual_noalloc"]


def default_params(**kw) -> Params:
    p = Params()
    N_.load().blp_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def mesh(N: int, eps: float, sigma: float = 2.0, beta: float = 1.0, graded: bool = False, parabolic: bool = False,
         layer_intervals: int | None = None):
    """Shishkin mesh nodes x[0..N] (blp_mesh) and the transition point tau;
    graded=True: the graded layer mesh with the same tau (blp_mesh_graded);
    parabolic=True: the parabolic-layer mesh, tau = min(1/2, sigma sqrt(eps)
    ln N) (blp_mesh_parabolic; beta is not used); layer_intervals=NL: the
    general Shishkin mesh with NL intervals on [0, tau] (blp_mesh_q)."""
    if graded + parabolic + (layer_intervals is not None) > 1:
        raise ValueError("graded, parabolic and layer_intervals are exclusive")
    x = np.zeros(N + 1)
    xp = x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if layer_intervals is not None:
        name, tau = "blp_mesh_q", N_.load().blp_mesh_q(N, int(layer_intervals), eps, sigma, beta, xp)
    elif parabolic:
        name, tau = "blp_mesh_parabolic", N_.load().blp_mesh_parabolic(N, eps, sigma, xp)
    else:
        name = "blp_mesh_graded" if graded else "blp_mesh"
        tau = getattr(N_.load(), name)(N, eps, sigma, beta, xp)
    if tau < 0:
        raise BlpError(N_.BLP_ERR_ARG, name)
    return x, tau


def _ptr(a, n, writable=False):
    """(pointer, keepalive) for a float64 contiguous array of n values."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n:
                raise ValueError(f"expected a contiguous float64 tensor of {n} values")
            return ctypes.c_void_p(a.data_ptr()), a
    except ImportError:
        pass
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != n:
        raise ValueError(f"expected a contiguous float64 array of {n} values")
    if writable and not a.flags["WRITEABLE"]:
        raise ValueError("output array is read-only")
    return ctypes.c_void_p(a.ctypes.data), a


class Solver:
    """One assembled problem on the current CUDA device (blp_setup)."""

    def __init__(self, N, eps, c1, c2, r, stream=None, **params):
        self.lib = N_.load()
        self.N = N
        self.n = (N - 1) ** 2
        self.params = default_params(N=N, eps=eps, **params)
        h = ctypes.c_void_p()
        self._h = None
        args = [_ptr(a, self.n)[0] for a in (c1, c2, r)]
        N_.check(self.lib.blp_setup(ctypes.byref(self.params), *args, ctypes.byref(h)), "blp_setup")
        self._h = h
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        if stream:
            N_.check(self.lib.blp_set_stream(h, ctypes.c_void_p(stream)), "blp_set_stream")

    def close(self):
        if self._h is not None:
            self.lib.blp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("solver closed")
        return self._h

    def _out_like(self, a):
        try:
            import torch
            if isinstance(a, torch.Tensor):
                return torch.zeros_like(a)
        except ImportError:
            pass
        return np.zeros(self.n)

    def solve(self, f, u=None, tol=1e-10, raise_on_noconv=True):
        """blp_solve.  u (optional) is the initial guess and is overwritten."""
        u = self._out_like(f) if u is None else u
        info = Info()
        st = self.lib.blp_solve(self.handle, _ptr(f, self.n)[0], _ptr(u, self.n, True)[0], tol, ctypes.byref(info))
        if st != N_.BLP_OK and (st != N_.BLP_ERR_NOCONV or raise_on_noconv):
            raise BlpError(st, "blp_solve")
        return u, info

    def solve_adjoint(self, g, lam=None, tol=1e-10, raise_on_noconv=True):
        lam = self._out_like(g) if lam is None else lam
        info = Info()
        st = self.lib.blp_solve_adjoint(self.handle, _ptr(g, self.n)[0], _ptr(lam, self.n, True)[0], tol,
                                        ctypes.byref(info))
        if st != N_.BLP_OK and (st != N_.BLP_ERR_NOCONV or raise_on_noconv):
            raise BlpError(st, "blp_solve_adjoint")
        return lam, info

    def grad(self, u, lam):
        outs = [self._out_like(u) for _ in range(3)]
        N_.check(self.lib.blp_grad(self.handle, _ptr(u, self.n)[0], _ptr(lam, self.n)[0],
                                   *[_ptr(o, self.n, True)[0] for o in outs]), "blp_grad")
        return tuple(outs)

    def apply(self, u, transpose=False):
        y = self._out_like(u)
        N_.check(self.lib.blp_apply_operator(self.handle, _ptr(u, self.n)[0], _ptr(y, self.n, True)[0],
                                             int(transpose)), "blp_apply_operator")
        return y

    def precond(self, v, transpose=False, precision=BLP_FP64):
        z = self._out_like(v)
        cyc = ctypes.c_int(0)
        N_.check(self.lib.blp_precond_apply(self.handle, _ptr(v, self.n)[0], _ptr(z, self.n, True)[0],
                                            int(transpose), int(precision), ctypes.byref(cyc)), "blp_precond_apply")
        return z, cyc.value

    def kernel_launches(self):
        return self.lib.blp_kernel_launches(self.handle)

    def tuning(self):
        """blp_get_tuning: the wavefront launch setting of this handle, as a
        dict (dts_chunk, dts_cluster, two_step, precond_ms)."""
        t = N_.Tuning()
        N_.check(self.lib.blp_get_tuning(self.handle, ctypes.byref(t)), "blp_get_tuning")
        return t.as_dict()

    def set_tuning(self, dts_chunk=None, dts_cluster=None, two_step=None):
        """blp_set_tuning: change some of the wavefront launch settings."""
        t = N_.Tuning()
        N_.check(self.lib.blp_get_tuning(self.handle, ctypes.byref(t)), "blp_get_tuning")
        for k, v in (("dts_chunk", dts_chunk), ("dts_cluster", dts_cluster), ("two_step", two_step)):
            if v is not None:
                setattr(t, k, int(v))
        N_.check(self.lib.blp_set_tuning(self.handle, ctypes.byref(t)), "blp_set_tuning")

    def autotune(self, precision=None, reps=3):
        """blp_autotune: time the preconditioner under every candidate
        wavefront setting, keep the fastest; returns it as a dict."""
        t = N_.Tuning()
        prec = self.params.precision if precision is None else precision
        N_.check(self.lib.blp_autotune(self.handle, int(prec), int(reps), ctypes.byref(t)), "blp_autotune")
        return t.as_dict()


def solve_batched(problems, tol=1e-10, concurrency=16, autotune=False):
    """blp_solve_batched: independent problems solved concurrently.

    problems: list of dicts with keys N, eps, c1, c2, r, f (float64 arrays or
    tensors of (N-1)**2 values, host or device), optional u (initial guess,
    overwritten with the solution) and any blp_params field.  autotune=True
    calls blp_solve_batched_tuned: wavefront launch settings tuned once per
    (N, precision) and cached for the process.  Returns a list of (u, Info);
    raises BlpError if any problem failed (the per-problem statuses are in
    the Info objects of the exception's .results)."""
    lib = N_.load()
    n = len(problems)
    items = (N_.BatchItem * n)()
    keep, outs = [], []
    for k, pr in enumerate(problems):
        pr = dict(pr)
        N, eps = pr.pop("N"), pr.pop("eps")
        nn = (N - 1) ** 2
        fields = [pr.pop(key) for key in ("c1", "c2", "r", "f")]
        u = pr.pop("u", None)
        if u is None:
            try:
                import torch
                u = torch.zeros_like(fields[3]) if isinstance(fields[3], torch.Tensor) else np.zeros(nn)
            except ImportError:
                u = np.zeros(nn)
        items[k].params = default_params(N=N, eps=eps, **pr)
        ptrs = [_ptr(a, nn) for a in fields] + [_ptr(u, nn, True)]
        keep.append(ptrs)
        items[k].c1, items[k].c2, items[k].r, items[k].f, items[k].u = [q[0] for q in ptrs]
        items[k].tol = tol
        outs.append(u)
    fn = lib.blp_solve_batched_tuned if autotune else lib.blp_solve_batched
    st = fn(items, n, int(concurrency))
    results = [(outs[k], items[k].info) for k in range(n)]
    if st != N_.BLP_OK:
        err = BlpError(st, "blp_solve_batched_tuned" if autotune else "blp_solve_batched")
        err.results = results
        raise err
    return results


def solve_1d_batched(problems, stream=None):
    """blp_solve_1d_batched: the 1D method of Sec. 2 (upwind scheme, Shishkin
    mesh, GMRES left-preconditioned with M of eq. (block_M), true-residual
    stop) for many problems at once, one GPU thread per problem.

    problems: dicts with N, eps, stop (absolute ||f - A u||_inf target) and
    c, r, f (device float64 tensors of N-1 values at the interior nodes of
    mesh(N, eps, sigma, c_low), i.e. the 1D Shishkin mesh with beta = c_low),
    optional c_low (default 1), sigma (default 2), maxit (default 64).
    Returns a list of (u, iters, resid, status); raises BlpError when a
    problem is invalid (nothing runs) and returns normally otherwise (check
    each status: BLP_ERR_NOCONV when maxit was reached)."""
    import torch
    lib = N_.load()
    n = len(problems)
    items = (N_.Problem1D * n)()
    outs, keep = [], []
    for k, pr in enumerate(problems):
        N = int(pr["N"])
        fields = [pr[key] for key in ("c", "r", "f")]
        # the output lives where f does; the library refuses anything but device arrays
        u = torch.zeros_like(fields[2]) if isinstance(fields[2], torch.Tensor) else np.zeros(N - 1)
        it = items[k]
        it.N, it.eps, it.stop = N, float(pr["eps"]), float(pr["stop"])
        it.c_low, it.sigma, it.maxit = float(pr.get("c_low", 1.0)), float(pr.get("sigma", 2.0)), int(pr.get("maxit", 64))
        ptrs = [_ptr(a, N - 1) for a in fields] + [_ptr(u, N - 1, True)]
        keep.append(ptrs)
        it.c, it.r, it.f, it.u = [q[0] for q in ptrs]
        outs.append(u)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.blp_solve_1d_batched(items, n, ctypes.c_void_p(stream))
    if st == N_.BLP_ERR_ARG:
        raise BlpError(st, "blp_solve_1d_batched (invalid problem: N even in [8, BLP_1D_MAX_N], 0 < eps <= 1, "
                           "c_low, sigma > 0, 1 <= maxit <= BLP_1D_MAXIT, device arrays)")
    if st not in (N_.BLP_OK, N_.BLP_ERR_NOCONV):
        N_.check(st, "blp_solve_1d_batched")
    return [(outs[k], items[k].iters, items[k].resid, items[k].status) for k in range(n)]


def residual_noalloc(N, x, y, eps, c1, c2, r, f, u, res=None, stream=None):
    """blp_residual_noalloc: residual f - A u and its norms, allocating no
    device memory and needing no Solver.

    For callers that cannot allocate device memory when they check a
    solution (memory fully reserved, or a path where cudaMalloc's device-wide
    synchronisation would stall other streams).  Every array must already be
    on the device: x, y the N+1 mesh nodes, the fields (N-1)**2 values; res
    (optional) receives f - A u.  Returns the host array
    [||s||, ||D^-1 s||, ||f||, ||D^-1 f||] (s = f - A u, D = diag(A)).
    N is limited to BLP_NOALLOC_MAX_N; calls on one device must not overlap.
    """
    if N > N_.BLP_NOALLOC_MAX_N:
        raise ValueError(f"N={N} exceeds the no-allocation limit N <= {N_.BLP_NOALLOC_MAX_N}")
    n = (N - 1) ** 2
    ptrs = [_ptr(a, N + 1)[0] for a in (x, y)] + [_ptr(a, n)[0] for a in (c1, c2, r, f, u)]
    rp = _ptr(res, n, True)[0] if res is not None else None
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    norms = np.zeros(4)
    st = N_.load().blp_residual_noalloc(N, ptrs[0], ptrs[1], float(eps), *ptrs[2:], rp,
                                        ctypes.c_void_p(norms.ctypes.data), ctypes.c_void_p(stream))
    if st == N_.BLP_ERR_ARG:
        raise BlpError(st, f"blp_residual_noalloc (N={N}: even, 8 <= N <= {N_.BLP_NOALLOC_MAX_N}; "
                           "0 < eps <= 1; every input on the device)")
    N_.check(st, "blp_residual_noalloc")
    return norms


def solve(f, c1, c2, r, N, eps, tol=1e-10, adjoint_tol=None, **params):
    """Differentiable solve u = A(c1, c2, r)^{-1} f (see autograd.BLPSolve).
    tol: forward tolerance; adjoint_tol: tolerance of the adjoint solve in the
    backward pass (default: tol)."""
    from .autograd import BLPSolve
    return BLPSolve.apply(f, c1, c2, r, N, eps, tol, adjoint_tol, params)

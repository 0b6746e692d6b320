"""One-dimensional oracle pieces (Sec. 2 of arXiv 2108.13468), numpy, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  These pin the 1D
analogue of the method against what the paper prints: the Shishkin mesh of
eq. (tau 1D), the upwind stencil eq. (stencil_1d), the block preconditioner
eq. (block_M), Theorems block_fact and big_bound, Table 1 (errors) and
Table 2 (GMRES iteration counts).

Table 2 was computed with MATLAB's ``gmres``, which applies its
preconditioner on the left (it runs GMRES on M^-1 A x = M^-1 b).  The
oracle's GMRES for that table therefore preconditions on the left, and
stops, as Sec. 2.5.1 states, on the true residual ||b - A x||_inf.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_banded


def mesh(N: int, eps: float, c_low: float, sigma: float = 2.0, q: float = 0.5):
    """Shishkin mesh, eq. (tau 1D); q != 1/2 is the general mesh of the remark
    on general Shishkin meshes (qN intervals in the layer)."""
    tau = min(q, sigma * eps / c_low * np.log(N))
    NL = int(round(q * N))
    x = np.empty(N + 1)
    x[: NL + 1] = np.arange(NL + 1) / NL * tau
    x[NL:] = tau + np.arange(N - NL + 1) / (N - NL) * (1.0 - tau)
    x[0], x[N] = 0.0, 1.0
    return x, tau, NL


def assemble(x: np.ndarray, eps: float, c, r):
    """Tridiagonal upwind matrix (eq. stencil_1d) on the interior nodes
    1..N-1: returns (sub, diag, sup) with c, r callables of x."""
    h = np.diff(x)                       # h[i-1] = h_i
    xi = x[1:-1]
    hi, hi1 = h[:-1], h[1:]
    hb = 0.5 * (hi + hi1)
    ci, ri = c(xi), r(xi)
    sub = -eps / (hi * hb)
    dia = eps / hb * (1.0 / hi + 1.0 / hi1) + ci / hi1 + ri
    sup = -eps / (hi1 * hb) - ci / hi1
    return sub, dia, sup


def dense(sub, dia, sup):
    n = dia.size
    A = np.diag(dia)
    A[np.arange(1, n), np.arange(n - 1)] = sub[1:]
    A[np.arange(n - 1), np.arange(1, n)] = sup[:-1]
    return A


def solve(sub, dia, sup, f):
    """Direct tridiagonal solve (LAPACK banded solver as the library step)."""
    n = dia.size
    ab = np.zeros((3, n))
    ab[0, 1:] = sup[:-1]
    ab[1] = dia
    ab[2, :-1] = sub[1:]
    return solve_banded((1, 1), ab, f)


def block_M(A: np.ndarray, NL: int) -> np.ndarray:
    """eq. (block_M): keep A_LL, A_LI, A_IL; replace A_II by its upper
    triangular part (diagonal included).  L = first NL unknowns (nodes
    1..NL, the transition node is node NL)."""
    M = A.copy()
    AII = M[NL:, NL:]
    M[NL:, NL:] = np.triu(AII)
    return M


def gmres_true_residual(A, b, M, stop, maxit=None):
    """Unrestarted GMRES, right preconditioned by M (dense), stopping on the
    true residual ||b - A x||_inf <= stop (the paper's modified stopping rule
    of Sec. 2.5.1).  Returns (x, iterations).  Table 2 uses the left
    preconditioned form below."""
    n = b.size
    maxit = maxit or n
    Minv = np.linalg.inv(M)
    x = np.zeros(n)
    r0 = b.copy()
    if np.abs(r0).max() <= stop:
        return x, 0
    beta = np.linalg.norm(r0)
    V = np.zeros((n, maxit + 1))
    H = np.zeros((maxit + 1, maxit))
    V[:, 0] = r0 / beta
    for j in range(maxit):
        w = A @ (Minv @ V[:, j])
        for i in range(j + 1):
            H[i, j] = w @ V[:, i]
            w -= H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] > 0:
            V[:, j + 1] = w / H[j + 1, j]
        e1 = np.zeros(j + 2)
        e1[0] = beta
        y = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)[0]
        x = Minv @ (V[:, : j + 1] @ y)
        if np.abs(b - A @ x).max() <= stop or H[j + 1, j] == 0:
            return x, j + 1
    return x, maxit


def gmres_left_true_residual(A, b, M, stop, maxit=None):
    """Unrestarted GMRES on the left-preconditioned system M^-1 A x = M^-1 b
    from x = 0: Arnoldi (modified Gram-Schmidt) on the Krylov space of M^-1 A
    started at M^-1 b, each iterate x_j = V_j y_j minimising ||M^-1 (b - A x)||_2
    over it, and the stop of Sec. 2.5.1 on the TRUE residual
    ||b - A x_j||_inf <= stop.  This is the setting of Table 2 (MATLAB's gmres,
    which preconditions on the left, with its stopping test replaced by the
    paper's).  Returns (x, iterations)."""
    n = b.size
    maxit = maxit or n
    Minv = np.linalg.inv(M)
    x = np.zeros(n)
    if np.abs(b).max() <= stop:
        return x, 0
    z0 = Minv @ b
    beta = np.linalg.norm(z0)
    V = np.zeros((n, maxit + 1))
    H = np.zeros((maxit + 1, maxit))
    V[:, 0] = z0 / beta
    for j in range(maxit):
        w = Minv @ (A @ V[:, j])
        for i in range(j + 1):
            H[i, j] = w @ V[:, i]
            w -= H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] > 0:
            V[:, j + 1] = w / H[j + 1, j]
        e1 = np.zeros(j + 2)
        e1[0] = beta
        y = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)[0]
        x = V[:, : j + 1] @ y
        if np.abs(b - A @ x).max() <= stop or H[j + 1, j] == 0:
            return x, j + 1
    return x, maxit

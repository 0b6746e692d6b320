"""Autotuned launch settings of the downstream sweeps (blp_autotune,
blp_set_tuning, blp_solve_batched_tuned) through the C ABI.

The settings reschedule the wavefront sweeps of Sec. 3.1 / 3.2 (hand-off
chunk, cluster size, one- or two-step recurrence) without changing what
they compute, so every tuned solve must keep the oracle parity of the
default one: FP64 path <= 1e-8, mixed path <= 1e-7 relative max-norm error
against the oracle's direct solve."""
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
    a = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def problem(N, eps, seed=0):
    x, _ = oracle.mesh(N, eps)
    p = inputs.problem_fourier_quadratic(x, x, N, eps, seed=seed)
    return p, oracle.assemble(N, eps, x, x, p.c1, p.c2, p.r)


@pytest.mark.parametrize("precision,tol", [(blp.BLP_FP64, 1e-8), (blp.BLP_MIXED, 1e-7)])
def test_autotune_picks_a_candidate_and_keeps_parity(precision, tol):
    N, eps = 256, 1e-4
    p, A = problem(N, eps)
    ue = oracle.band_solve(N, A, p.f)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r), precision=precision)
    t = s.autotune()
    # N = 256: 4-strip blocks, so the candidate clusters are 2 and 4
    assert t["dts_chunk"] in (8, 16, 32) and t["dts_cluster"] in (2, 4) and 0 <= t["two_step"] <= 3
    assert t["precond_ms"] > 0.0 and s.tuning() == t
    u, info = s.solve(T(p.f), tol=1e-10)
    assert info.status == 0 and rel(u, ue) <= tol


def test_set_tuning_validates_and_every_setting_solves():
    N, eps = 130, 1e-6
    p, A = problem(N, eps, seed=1)
    ue = oracle.band_solve(N, A, p.f)
    s = blp.Solver(N, eps, T(p.c1), T(p.c2), T(p.r))
    assert s.tuning()["precond_ms"] == -1.0
    for bad in (dict(dts_chunk=12), dict(dts_cluster=0), dict(dts_cluster=17), dict(two_step=4)):
        with pytest.raises(blp.BlpError) as e:
            s.set_tuning(**bad)
        assert e.value.status == _native.BLP_ERR_ARG
    u0, _ = s.solve(T(p.f), tol=1e-10)   # default setting (captures its graphs)
    for chunk, cluster, two in ((8, 1, 3), (32, 2, 0), (16, 16, 1)):
        s.set_tuning(dts_chunk=chunk, dts_cluster=cluster, two_step=two)   # drops the captured graphs
        assert s.tuning()["dts_chunk"] == chunk and s.tuning()["dts_cluster"] == cluster
        for _ in range(2):   # eager application, then a graph captured under the new setting
            u, info = s.solve(T(p.f), tol=1e-10)
            assert info.status == 0 and rel(u, ue) <= 1e-8
            if not two & 2:   # FP64 one-step form: chunk and cluster change no arithmetic at all
                assert torch.equal(u, u0)


def test_batched_tuned_matches_direct_solves():
    specs = [(64, 1e-2, blp.BLP_MIXED), (96, 1e-8, blp.BLP_FP64), (130, 1e-4, blp.BLP_MIXED), (130, 1e-6, blp.BLP_MIXED),
             (96, 1e-3, blp.BLP_FP64), (64, 1e-5, blp.BLP_MIXED)]
    probs, want = [], []
    for k, (N, eps, prec) in enumerate(specs):
        p, A = problem(N, eps, seed=k)
        want.append(oracle.band_solve(N, A, p.f))
        probs.append(dict(N=N, eps=eps, c1=T(p.c1), c2=T(p.c2), r=T(p.r), f=T(p.f), precision=prec, maxit=3000))
    res = blp.solve_batched(probs, tol=1e-10, concurrency=3, autotune=True)
    for (N, eps, prec), (u, info), w in zip(specs, res, want):
        assert info.status == 0 and rel(u, w) <= (1e-8 if prec == blp.BLP_FP64 else 1e-7), (N, eps)
    # a second call reuses the cached settings and gives the same answers
    res2 = blp.solve_batched(probs, tol=1e-10, concurrency=2, autotune=True)
    for (u, _), (u2, _) in zip(res, res2):
        assert rel(u2, u.cpu().numpy()) <= 1e-12

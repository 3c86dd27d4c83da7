"""Factorized CR through the C ABI (sylv_cr) against the CPU oracle.

Sec. 4 names CR among the methods the factorized approach carries over to; the oracle's
factorized CR is pinned (tests/test_oracle_pins.py) to the matrix-oriented recurrence, to
scipy's MINRES on the Kronecker system (same iterates for a self-adjoint operator) and to the
Bartels-Stewart solution.  The GPU must match it to 1e-10 relative Frobenius error of
X = V X^ W^T at fixed iteration counts (several tiles, ragged tails, s = 1..5, Sylvester and
Lyapunov forms), converge to the same solution, and in the mixed mode reach the stated true
residual through refinement rounds that also run CR.
"""
import ctypes

import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl
from oracle import exact, factorized as fz, residual

pytestmark = pytest.mark.gpu

TOL_X = 1e-10
STOP_MARGIN = 0.4  # default sylv_options.stop_margin: the recurrence test of a certified FP64 solve


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_cr(A, B, C1, C2, tol, maxit, lyapunov=False, **kw):
    with ps.Solver(A, None if lyapunov else B, C1, None if lyapunov else C2, lyapunov=lyapunov, **kw) as sv:
        info = sv.cr(tol, maxit)
        V, Xh, W = sv.factors()
        hist = sv.history()
    return info, V, Xh, W, hist


@pytest.mark.parametrize("NA,NB,s", [(17, 13, 1), (20, 11, 3), (12, 9, 5)])
def test_cr_matches_oracle_at_fixed_iterations(NA, NB, s):
    A, B = wl.laplacian_2d(NA, 0.1), wl.laplacian_2d(NB)
    C1, C2 = wl.rhs(A.nrows, B.nrows, s, 0)
    for maxit in (1, 3, 12):
        info, V, Xh, W, hist = gpu_cr(A, B, C1, C2, 0.0, maxit)
        ref = fz.factorized_cr(A.to_scipy(), B.to_scipy(), C1, C2, 0.0, maxit)
        assert info["iters"] == maxit and info["width"] == maxit * s, info
        assert info["matvecs"] == maxit + 1
        assert rel(V @ Xh @ W.T, ref.X()) < TOL_X
        np.testing.assert_allclose(hist, ref.history, rtol=1e-8)


def test_cr_ragged_random_spd_matches_oracle():
    A = wl.random_sparse(700, 3, 21, spd=True)
    B = wl.random_sparse(333, 4, 22, spd=True)
    C1, C2 = wl.rhs(700, 333, 2, 1)
    for maxit in (2, 9):
        info, V, Xh, W, hist = gpu_cr(A, B, C1, C2, 0.0, maxit)
        ref = fz.factorized_cr(A.to_scipy(), B.to_scipy(), C1, C2, 0.0, maxit)
        assert rel(V @ Xh @ W.T, ref.X()) < TOL_X


def test_lyapunov_cr_matches_oracle_and_is_symmetric():
    A = wl.laplacian_2d(16, 0.5)
    C1, _ = wl.rhs(A.nrows, None, 3, 2)
    for maxit in (2, 10):
        info, V, Xh, W, hist = gpu_cr(A, None, C1, None, 0.0, maxit, lyapunov=True)
        ref = fz.factorized_cr(A.to_scipy(), None, C1, None, 0.0, maxit, lyapunov=True)
        assert rel(V @ Xh @ W.T, ref.X()) < TOL_X
        assert np.abs(Xh - Xh.T).max() <= 1e-13 * np.abs(Xh).max()


def test_cr_converges_like_oracle():
    A, B = wl.laplacian_2d(20, 0.1), wl.laplacian_2d(14)
    C1, C2 = wl.rhs(A.nrows, B.nrows, 2, 0)
    info, V, Xh, W, hist = gpu_cr(A, B, C1, C2, 1e-8, 400)
    ref = fz.factorized_cr(A.to_scipy(), B.to_scipy(), C1, C2, 1e-8 * STOP_MARGIN, 400)
    assert info["status"] == ps.SYLV_OK and ref.status == "converged"
    assert abs(info["iters"] - ref.iters) <= 2
    Xe = exact.bartels_stewart(A.to_dense(), B.to_dense(), C1 @ C2.T)
    X = V @ Xh @ W.T
    assert rel(X, ref.X()) < max(TOL_X, 10 * rel(ref.X(), Xe))
    assert rel(X, Xe) < 1e-6
    assert info["true_rel_bound"] <= 1e-8
    assert residual.direct(A.to_scipy(), B.to_scipy(), C1, C2, V, Xh, W) <= 1e-8 * np.linalg.norm(C1 @ C2.T)


def test_mixed_cr_reaches_true_residual():
    A, B = wl.laplacian_2d(60, 0.05), wl.laplacian_2d(45)
    C1, C2 = wl.rhs(A.nrows, B.nrows, 4, 0)
    info, V, Xh, W, _ = gpu_cr(A, B, C1, C2, 1e-8, 400, precision="mixed")
    t = residual.direct(A.to_scipy(), B.to_scipy(), C1, C2, V, Xh, W) / np.linalg.norm(C1 @ C2.T)
    assert info["status"] == ps.SYLV_OK, info
    assert t <= 1e-8, (t, info)
    assert t <= info["true_rel_bound"] <= 1e-8, (t, info)
    assert abs(info["true_rel_res"] - t) <= 0.2 * t


def test_cr_rejected_on_batched_handle():
    probs = wl.cfg_batched_lyapunov(count=2, seed=5)
    with ps.BatchSolver([q.A for q in probs], [q.C1 for q in probs]) as bs:
        info = ps.sylv_info()
        assert ps.load().sylv_cr(bs.h, 1e-8, 10, ctypes.byref(info)) == ps.SYLV_EINVAL

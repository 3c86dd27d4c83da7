"""Factorized CGS through the C ABI (sylv_cgs) against the CPU oracle.

Sec. 4 names CGS among the methods the factorized approach carries over to; the oracle's
factorized CGS is pinned (tests/test_oracle_pins.py) to the matrix-oriented recurrence, to
scipy's CGS on the Kronecker system and to the Bartels-Stewart solution.  The GPU must
match it to 1e-10 relative Frobenius error of X = V X^ W^T at fixed iteration counts
(several tiles, ragged tails, s = 1..5), converge to the same solution, and in the mixed
mode reach the stated true residual through refinement rounds that also run CGS.
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


def gpu_cgs(A, B, C1, C2, tol, maxit, **kw):
    with ps.Solver(A, B, C1, C2, **kw) as sv:
        info = sv.cgs(tol, maxit)
        V, Xh, W = sv.factors()
        hist = sv.history()
    return info, V, Xh, W, hist


@pytest.mark.parametrize("NA,NB,s", [(9, 7, 2), (10, 8, 5), (11, 5, 1)])
@pytest.mark.parametrize("small_gemm", [1, 2])
def test_cgs_matches_oracle_at_fixed_iterations(NA, NB, s, small_gemm):
    A, B = wl.convdiff_3d(NA, 1), wl.convdiff_3d(NB, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, s, 0)
    for maxit in (1, 3, 10):
        info, V, Xh, W, hist = gpu_cgs(A, B, C1, C2, 0.0, maxit, small_gemm=small_gemm)
        ref = fz.factorized_cgs(A.to_scipy(), B.to_scipy(), C1, C2, 0.0, maxit)
        assert info["iters"] == maxit and info["width"] == 2 * maxit * s, info
        assert rel(V @ Xh @ W.T, ref.X()) < TOL_X
        np.testing.assert_allclose(hist, ref.history, rtol=1e-8)


@pytest.mark.parametrize("NA,NB,s", [(9, 7, 2), (12, 10, 4)])
def test_cgs_converges_like_oracle(NA, NB, s):
    A, B = wl.convdiff_3d(NA, 1), wl.convdiff_3d(NB, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, s, 0)
    info, V, Xh, W, hist = gpu_cgs(A, B, C1, C2, 1e-8, 300)
    ref = fz.factorized_cgs(A.to_scipy(), B.to_scipy(), C1, C2, 1e-8 * STOP_MARGIN, 300)
    assert info["status"] == ps.SYLV_OK and ref.status == "converged"
    assert abs(info["iters"] - ref.iters) <= max(2, ref.iters // 10)
    np.testing.assert_allclose(hist[:11], ref.history[:11], rtol=1e-7)
    Xe = exact.bartels_stewart(A.to_dense(), B.to_dense(), C1 @ C2.T)
    X = V @ Xh @ W.T
    assert rel(X, ref.X()) < max(TOL_X, 10 * rel(ref.X(), Xe))
    assert rel(X, Xe) < 1e-6
    assert info["true_rel_bound"] <= 1e-8
    assert residual.direct(A.to_scipy(), B.to_scipy(), C1, C2, V, Xh, W) <= 1e-8 * np.linalg.norm(C1 @ C2.T)


def test_mixed_cgs_reaches_true_residual():
    A, B = wl.convdiff_3d(13, 1), wl.convdiff_3d(9, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, 3, 0)
    info, V, Xh, W, _ = gpu_cgs(A, B, C1, C2, 1e-8, 300, precision="mixed")
    t = residual.direct(A.to_scipy(), B.to_scipy(), C1, C2, V, Xh, W) / np.linalg.norm(C1 @ C2.T)
    assert info["status"] == ps.SYLV_OK, info
    assert t <= 1e-8, (t, info)
    assert t <= info["true_rel_bound"] <= 1e-8, (t, info)
    assert abs(info["true_rel_res"] - t) <= 0.2 * t


def test_cgs_rejected_on_batched_handle():
    probs = wl.cfg_batched_lyapunov(count=2, seed=5)
    with ps.BatchSolver([q.A for q in probs], [q.C1 for q in probs]) as bs:
        info = ps.sylv_info()
        assert ps.load().sylv_cgs(bs.h, 1e-8, 10, ctypes.byref(info)) == ps.SYLV_EINVAL

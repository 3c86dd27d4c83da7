"""The small Sylvester operator of BiCGSTAB, Q^ = [H P^, 0] + [P^ G^T; 0] (eq. 3.7), on the
tcgen05 tensor cores: both factors split exactly into BF16 digits (Ozaki scheme I), FP32
accumulation in tensor memory, double-float folds, float64 accuracy.

small_gemm = 2 forces the tensor-core form at every order (the default switches to it from
r = 448 on).  It must keep the FP64 parity bar against the oracle (1e-10 relative Frobenius
error of X = V X^ W^T at fixed iteration counts, spanning several 128 x 64 output tiles and
ragged tails), follow the CUDA-core float64 operator iterate by iterate, and, in the mixed
mode, still reach the stated true residual.
"""
import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl
from oracle import exact, factorized as fz, residual

pytestmark = pytest.mark.gpu

TOL_X = 1e-10


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solve(A, B, C1, C2, tol, maxit, precision="fp64", **kw):
    with ps.Solver(A, B, C1, C2, precision=precision, **kw) as sv:
        info = sv.bicgstab(tol, maxit)
        V, Xh, W = sv.factors()
        hist = sv.history()
    return info, V, Xh, W, hist


@pytest.mark.parametrize("NA,NB,s", [(9, 7, 2), (10, 8, 5), (11, 5, 1), (12, 10, 4)])
def test_tensor_small_side_matches_oracle_at_fixed_iterations(NA, NB, s):
    A, B = wl.convdiff_3d(NA, 1), wl.convdiff_3d(NB, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, s, 0)
    for maxit in (1, 3, 17):
        info, V, Xh, W, hist = solve(A, B, C1, C2, 0.0, maxit, small_gemm=2)
        ref = fz.factorized_bicgstab(A.to_scipy(), B.to_scipy(), C1, C2, 0.0, maxit)
        if ref.status == "breakdown":
            continue
        assert info["iters"] == maxit, info
        assert rel(V @ Xh @ W.T, ref.X()) < TOL_X
        np.testing.assert_allclose(hist, ref.history, rtol=1e-8)


@pytest.mark.parametrize("NA,NB,s", [(12, 10, 4), (14, 9, 3)])
def test_tensor_small_side_follows_fp64_operator_to_convergence(NA, NB, s):
    A, B = wl.convdiff_3d(NA, 1), wl.convdiff_3d(NB, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, s, 0)
    i2, V2, X2, W2, h2 = solve(A, B, C1, C2, 1e-8, 300, small_gemm=2)
    i1, V1, X1, W1, h1 = solve(A, B, C1, C2, 1e-8, 300, small_gemm=1)
    assert i2["status"] == ps.SYLV_OK and i1["status"] == ps.SYLV_OK
    assert abs(i2["iters"] - i1["iters"]) <= 1
    k = min(len(h1), len(h2), 30)
    # the two operators round differently; BiCGSTAB amplifies that, so late entries agree to ~1e-11
    np.testing.assert_allclose(h2[:k], h1[:k], rtol=1e-6, atol=1e-10)
    ref = fz.factorized_bicgstab(A.to_scipy(), B.to_scipy(), C1, C2, 1e-8, 300)
    Xe = exact.bartels_stewart(A.to_dense(), B.to_dense(), C1 @ C2.T)
    X = V2 @ X2 @ W2.T
    assert rel(X, ref.X()) < max(TOL_X, 10 * rel(ref.X(), Xe))
    assert rel(X, V1 @ X1 @ W1.T) < max(TOL_X, 10 * rel(ref.X(), Xe))
    assert i2["true_rel_bound"] <= 1e-8
    assert residual.direct(A.to_scipy(), B.to_scipy(), C1, C2, V2, X2, W2) <= 1e-8 * np.linalg.norm(C1 @ C2.T)


def test_mixed_mode_with_tensor_small_side_reaches_true_residual():
    A, B = wl.convdiff_3d(16, 1), wl.convdiff_3d(12, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, 4, 0)
    info, V, Xh, W, _ = solve(A, B, C1, C2, 1e-8, 300, precision="mixed", small_gemm=2)
    t = residual.direct(A.to_scipy(), B.to_scipy(), C1, C2, V, Xh, W) / np.linalg.norm(C1 @ C2.T)
    assert info["status"] == ps.SYLV_OK, info
    assert t <= 1e-8, (t, info)
    assert t <= info["true_rel_bound"] <= 1e-8, (t, info)
    assert abs(info["true_rel_res"] - t) <= 0.2 * t

"""Partial loss of rank in a basis block (0 < rank < s): the dependent columns are deflated to
zero basis columns (CholQR pivot <= delta * nu), exactly as the oracle's Gram-Schmidt QR drops
them, instead of stopping with SYLV_EBREAKDOWN.  C1 = [c, A c, ...] makes one column of every
basis block after the first dependent.  The GPU must match the oracle (1e-10 on X at fixed
iteration counts), converge to the Bartels-Stewart solution with every method, and return a
basis whose deflated columns are zero."""
import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl
from oracle import exact, factorized as fz

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def arnoldi_problem():
    A, B = wl.convdiff_3d(6, 1), wl.convdiff_3d(5, 2)
    rng = np.random.default_rng(3)
    c = rng.standard_normal(A.nrows)
    C1 = np.column_stack([c, A.to_scipy() @ c, rng.standard_normal(A.nrows)])
    C2 = rng.standard_normal((B.nrows, 3))
    return A, B, C1, C2


def lanczos_problem():
    A, B = wl.laplacian_2d(8), wl.laplacian_2d(7)
    rng = np.random.default_rng(4)
    c = rng.standard_normal(A.nrows)
    return A, B, np.column_stack([c, A.to_scipy() @ c]), rng.standard_normal((B.nrows, 2))


@pytest.mark.parametrize("method", ["bicgstab", "cgs", "gpbicg"])
def test_arnoldi_methods_deflate_like_oracle(method):
    A, B, C1, C2 = arnoldi_problem()
    oracle = getattr(fz, "factorized_" + method)
    for maxit in (2, 6):
        with ps.Solver(A, B, C1, C2) as sv:
            info = getattr(sv, method)(0.0, maxit)
            V, Xh, W = sv.factors()
        ref = oracle(A.to_scipy(), B.to_scipy(), C1, C2, 0.0, maxit)
        assert info["iters"] == maxit, info
        assert rel(V @ Xh @ W.T, ref.X()) < 1e-10
        zero_gpu = np.linalg.norm(V, axis=0) == 0.0
        zero_ref = np.linalg.norm(ref.V, axis=0) == 0.0
        assert zero_gpu.any() and (zero_gpu == zero_ref).all()
    with ps.Solver(A, B, C1, C2) as sv:
        info = getattr(sv, method)(1e-10, 300)
        V, Xh, W = sv.factors()
    assert info["status"] == ps.SYLV_OK, info
    assert rel(V @ Xh @ W.T, exact.bartels_stewart(A.to_dense(), B.to_dense(), C1 @ C2.T)) < 1e-8


@pytest.mark.parametrize("method", ["cg", "cr"])
def test_lanczos_methods_deflate_like_oracle(method):
    A, B, C1, C2 = lanczos_problem()
    oracle = getattr(fz, "factorized_" + method)
    with ps.Solver(A, B, C1, C2) as sv:
        info = getattr(sv, method)(0.0, 5)
        V, Xh, W = sv.factors()
    ref = oracle(A.to_scipy(), B.to_scipy(), C1, C2, 0.0, 5)
    assert rel(V @ Xh @ W.T, ref.X()) < 1e-10
    with ps.Solver(A, B, C1, C2) as sv:
        info = getattr(sv, method)(1e-10, 300)
        V, Xh, W = sv.factors()
    assert info["status"] == ps.SYLV_OK, info
    assert rel(V @ Xh @ W.T, exact.bartels_stewart(A.to_dense(), B.to_dense(), C1 @ C2.T)) < 1e-8


def test_mixed_mode_deflates_and_reaches_true_residual():
    A, B, C1, C2 = arnoldi_problem()
    with ps.Solver(A, B, C1, C2, precision="mixed") as sv:
        info = sv.bicgstab(1e-8, 300)
    assert info["status"] == ps.SYLV_OK, info
    assert info["true_rel_res"] <= info["true_rel_bound"] <= 1e-8, info

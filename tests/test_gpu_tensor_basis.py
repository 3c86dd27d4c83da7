"""Float64 block Gram products and block updates of the Arnoldi bases on the tcgen05 tensor
cores (sylv_options.basis_gemm; the default of FP64 BiCGSTAB, CGS and GPBiCG).  Each basis
block is kept, once built, as seven BF16 planes of 8-bit digits (56 bits on its column's
scale); the other operand is split the same way; sums of digit products are exact integers,
rounded once to float64 (Ozaki scheme I).

Against the CPU oracle: X = V X^ W^T to 1e-10 relative Frobenius error and the residual
history at fixed iteration counts, and the block Hessenberg matrix of eq. 3.4, for block
widths s = 1..8 (every MMA width, both tensor-memory sizes), bases wider than one 128-column
tile, Gram products split over many CTAs, update row tiles several per CTA, and ragged row
counts.  Against the CUDA-core float64 kernels (basis_gemm = 1): the same convergence for
BiCGSTAB, CGS and GPBiCG.  At any size: orthonormality of V and the Arnoldi relation.
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


def solve(A, B, C1, C2, tol, maxit, method="bicgstab", **kw):
    with ps.Solver(A, B, C1, C2, **kw) as sv:
        info = getattr(sv, method)(tol, maxit)
        V, Xh, W = sv.factors()
        hist = sv.history()
        H = sv.hessenberg(0)
    return info, V, Xh, W, hist, H


@pytest.mark.parametrize("NA,NB,s", [(9, 7, 2), (10, 8, 5), (11, 5, 1), (12, 10, 4), (8, 6, 3), (9, 8, 6),
                                     (8, 7, 7), (8, 8, 8)])
def test_tensor_basis_matches_oracle_at_fixed_iterations(NA, NB, s):
    A, B = wl.convdiff_3d(NA, 1), wl.convdiff_3d(NB, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, s, 0)
    for maxit in (1, 3, 17):
        info, V, Xh, W, hist, H = solve(A, B, C1, C2, 0.0, maxit, basis_gemm=2)
        ref = fz.factorized_bicgstab(A.to_scipy(), B.to_scipy(), C1, C2, 0.0, maxit)
        if ref.status == "breakdown":
            continue
        assert info["iters"] == maxit and info["width"] == 2 * maxit * s, info
        assert rel(V @ Xh @ W.T, ref.X()) < TOL_X
        np.testing.assert_allclose(hist, ref.history, rtol=1e-8)
        if maxit <= 3:
            assert rel(H, ref.basisA.Hk(2 * maxit + 1, 2 * maxit)) < 1e-12


@pytest.mark.parametrize("NA,NB,s,maxit", [(24, 12, 4, 17), (40, 12, 2, 3)])
def test_tensor_basis_large_rows_match_oracle(NA, NB, s, maxit):
    # n = 13,824: 144 Gram splits of several folds; n = 64,000: 500 update row tiles, 3-4 per CTA
    A, B = wl.convdiff_3d(NA, 1), wl.convdiff_3d(NB, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, s, 0)
    info, V, Xh, W, hist, H = solve(A, B, C1, C2, 0.0, maxit, basis_gemm=2)
    ref = fz.factorized_bicgstab(A.to_scipy(), B.to_scipy(), C1, C2, 0.0, maxit)
    assert info["iters"] == maxit
    assert rel(V @ Xh @ W.T, ref.X()) < TOL_X
    np.testing.assert_allclose(hist, ref.history, rtol=1e-8)


@pytest.mark.parametrize("method", ["bicgstab", "cgs", "gpbicg"])
def test_tensor_basis_follows_fp64_kernels_to_convergence(method):
    A, B = wl.convdiff_3d(14, 1), wl.convdiff_3d(9, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, 3, 0)
    i2, V2, X2, W2, h2, _ = solve(A, B, C1, C2, 1e-8, 300, method, basis_gemm=2)
    i1, V1, X1, W1, h1, _ = solve(A, B, C1, C2, 1e-8, 300, method, basis_gemm=1)
    assert i2["status"] == ps.SYLV_OK and i1["status"] == ps.SYLV_OK, (i2, i1)
    assert abs(i2["iters"] - i1["iters"]) <= max(2, i1["iters"] // 10)
    k = min(len(h1), len(h2), 11)
    np.testing.assert_allclose(h2[:k], h1[:k], rtol=1e-7)
    Xe = exact.bartels_stewart(A.to_dense(), B.to_dense(), C1 @ C2.T)
    X2f = V2 @ X2 @ W2.T
    assert rel(X2f, Xe) < 1e-6
    assert rel(X2f, V1 @ X1 @ W1.T) < max(TOL_X, 10 * rel(V1 @ X1 @ W1.T, Xe))
    assert i2["true_rel_bound"] <= 1e-8
    assert residual.direct(A.to_scipy(), B.to_scipy(), C1, C2, V2, X2, W2) <= 1e-8 * np.linalg.norm(C1 @ C2.T)


def test_tensor_basis_orthonormal_and_arnoldi_relation():
    # 61 iterations at s = 4: 496 basis columns (four 128-column tiles), 27,000 rows
    A, B = wl.convdiff_3d(30, 1), wl.convdiff_3d(10, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, 4, 0)
    info, V, Xh, W, hist, H = solve(A, B, C1, C2, 0.0, 61, basis_gemm=2)
    assert info["iters"] == 61
    w = V.shape[1]
    assert np.abs(V.T @ V - np.eye(w)).max() < 1e-12
    As = A.to_scipy()
    lhs = As @ V[:, : w - 4]
    rhs = V @ H[:w, : w - 4]
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max() * 10


def test_basis_gemm_modes_agree_on_one_handle():
    A, B = wl.convdiff_3d(9, 1), wl.convdiff_3d(7, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, 2, 0)
    out = {}
    for mode in (0, 1, 2):
        with ps.Solver(A, B, C1, C2, basis_gemm=mode) as sv:
            sv.bicgstab(0.0, 5)
            V, Xh, W = sv.factors()
            out[mode] = V @ Xh @ W.T
            sv.cg(1e-6, 50)  # Lanczos bases keep the CUDA-core kernels on the same handle
            sv.bicgstab(0.0, 5)
            V, Xh, W = sv.factors()
            assert rel(V @ Xh @ W.T, out[mode]) < 1e-13
    assert rel(out[0], out[1]) < TOL_X and rel(out[2], out[1]) < TOL_X

"""Final low-rank compression (sylv_compress) against the oracle's SVD-based compression.

The oracle compresses the GPU's own uncompressed factors (numpy SVD of X^, the same rank rule),
which isolates the compression step: the same rank q, the same singular values, the same
rank-q matrix X_q = V_q diag(s_q) W_q^T, orthonormal compressed factors, and the
Eckart-Young error.  Sizes span several Jacobi rounds and GEMM tiles with ragged tails.
"""
import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl
from oracle import compress

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("method", ["bicgstab", "gpbicg", "cgs"])
@pytest.mark.parametrize("tol", [1e-2, 1e-6, 1e-10])
def test_compression_matches_oracle(method, tol):
    A, B = wl.convdiff_3d(10, 1), wl.convdiff_3d(8, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, 3, 0)
    with ps.Solver(A, B, C1, C2) as sv:
        info = getattr(sv, method)(1e-10, 300)
        assert info["status"] == ps.SYLV_OK
        V, Xh, W = sv.factors()
        q = sv.compress(tol)
        Vq, Xq_hat, Wq = sv.factors()
    X = V @ Xh @ W.T
    Vo, so, Wo = compress.compress(V, Xh, W, tol)
    assert q == len(so) and Vq.shape == (A.nrows, q) and Wq.shape == (B.nrows, q)
    np.testing.assert_allclose(np.diag(Xq_hat), so, rtol=1e-9, atol=1e-12 * so[0])
    Xq = Vq @ Xq_hat @ Wq.T
    assert np.linalg.norm(Xq - (Vo * so) @ Wo.T) <= 1e-10 * np.linalg.norm(X)
    assert np.abs(Vq.T @ Vq - np.eye(q)).max() < 1e-10
    assert np.abs(Wq.T @ Wq - np.eye(q)).max() < 1e-10
    sx = np.linalg.svd(Xh, compute_uv=False)
    assert abs(np.linalg.norm(X - Xq) - np.sqrt(np.sum(sx[q:] ** 2))) <= 1e-9 * np.linalg.norm(X)


def test_compression_rules():
    A, B = wl.convdiff_3d(8, 1), wl.convdiff_3d(6, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, 2, 0)
    with ps.Solver(A, B, C1, C2) as sv:
        with pytest.raises(ps.SylvError) as e:
            sv.compress(1e-6)  # no solve yet
        assert e.value.code == ps.SYLV_ESTATE
        sv.bicgstab(1e-8, 300)
        r = sv.factors()[1].shape[0]
        assert sv.compress(0.0) <= r
        with pytest.raises(ps.SylvError) as e:
            sv.compress(1e-6)  # already compressed
        assert e.value.code == ps.SYLV_ESTATE
        sv.bicgstab(1e-8, 300)  # a new solve drops the compressed factors
        assert sv.factors()[1].shape[0] == r
        assert sv.compress(1.0) == 0
        sv.cg(1e-8, 300)
        with pytest.raises(ps.SylvError) as e:
            sv.compress(1e-6)  # Lanczos bases are not orthonormal
        assert e.value.code == ps.SYLV_EINVAL
    with ps.Solver(A, B, C1, C2, precision="mixed") as sv:
        sv.bicgstab(1e-8, 300)
        with pytest.raises(ps.SylvError) as e:
            sv.compress(1e-6)
        assert e.value.code == ps.SYLV_EINVAL

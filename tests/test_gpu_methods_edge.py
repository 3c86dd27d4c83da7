"""Edge cases of the CGS, CR and GPBiCG entry points (the methods Sec. 4 names beyond
Algorithms 4.1/4.2): zero iterations, every method in turn on one handle (device buffers
reallocated or reused between methods), a rank-deficient right-hand side factor, and block
Krylov spaces that fill up (the factorized iterate then reaches the exact solution)."""
import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl
from oracle import exact

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("method", ["cgs", "cr", "gpbicg"])
def test_zero_iterations(method):
    A = wl.laplacian_2d(10)
    C1, C2 = wl.rhs(100, 100, 2, 0)
    with ps.Solver(A, A, C1, C2) as sv:
        info = getattr(sv, method)(1e-8, 0)
        assert info["status"] == ps.SYLV_ENOTCONV and info["width"] == 0


def test_all_methods_on_one_handle_agree():
    A, B = wl.laplacian_2d(12, 0.3), wl.laplacian_2d(9, 0.3)
    C1, C2 = wl.rhs(144, 81, 3, 1)
    Xe = exact.bartels_stewart(A.to_dense(), B.to_dense(), C1 @ C2.T)
    with ps.Solver(A, B, C1, C2) as sv:
        for method in ("bicgstab", "cgs", "gpbicg", "cr", "cg", "gpbicg", "cgs"):
            info = getattr(sv, method)(1e-10, 300)
            assert info["status"] == ps.SYLV_OK, (method, info)
            V, Xh, W = sv.factors()
            assert rel(V @ Xh @ W.T, Xe) < 1e-7, method


@pytest.mark.parametrize("method", ["cgs", "cr", "gpbicg"])
def test_rank_deficient_rhs_breaks_down(method):
    A = wl.laplacian_2d(10)
    C1, C2 = wl.rhs(100, 100, 2, 0)
    with ps.Solver(A, A, np.ones((100, 2)), C2) as sv:
        assert getattr(sv, method)(1e-8, 10)["status"] == ps.SYLV_EBREAKDOWN


@pytest.mark.parametrize("method", ["cgs", "gpbicg", "cr"])
def test_exhausted_block_krylov_space_reaches_exact(method):
    n, s = 12, 3  # both block Krylov spaces fill up after 4 blocks
    A = wl.random_sparse(n, 2, 41, spd=True)
    B = wl.random_sparse(n, 2, 42, spd=True)
    C1, C2 = wl.rhs(n, n, s, 1)
    with ps.Solver(A, B, C1, C2) as sv:
        info = getattr(sv, method)(1e-12, 100)
        V, Xh, W = sv.factors()
    assert info["status"] == ps.SYLV_OK, info
    X = exact.kron_solve(A.to_dense(), B.to_dense(), C1 @ C2.T)
    assert rel(V @ Xh @ W.T, X) < 1e-9


def test_host_timeout_returns_etimeout_and_handle_stays_usable():
    # The host's wall-clock limit (sylv_options.timeout_s, SYLV_ETIMEOUT): a solve of about a
    # hundred milliseconds under a 0.1 ms limit gives up at its first status poll and returns
    # without waiting for the kernels it enqueued.  The same handle, with the limit raised, then
    # solves again and matches the oracle.
    from oracle import factorized as fz

    A, B = wl.convdiff_3d(40, 1), wl.convdiff_3d(30, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, 4, 0)
    with ps.Solver(A, B, C1, C2, timeout_s=1e-4) as sv:
        info = sv.bicgstab(0.0, 80)
        assert info["status"] == ps.SYLV_ETIMEOUT, info
        assert "timeout" in ps.last_error()
        sv.set_timeout(600.0)
        info = sv.bicgstab(0.0, 3)
        assert info["status"] == ps.SYLV_ENOTCONV and info["iters"] == 3, info
        V, Xh, W = sv.factors()
    ref = fz.factorized_bicgstab(A.to_scipy(), B.to_scipy(), C1, C2, 0.0, 3)
    assert rel(V @ Xh @ W.T, ref.X()) < 1e-10

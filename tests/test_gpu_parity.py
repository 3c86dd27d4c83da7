"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

FP64 mode: the factored solution X = V X^ W^T must match the oracle's to a
relative Frobenius error of 1e-10 (the stated bar), the residual histories must
agree iteration by iteration, and the block Hessenberg matrices (unique under
the diag(R) > 0 convention) must match while the bases are still orthonormal.
A default (certified) solve runs the printed recurrence test at STOP_MARGIN * tol,
so it is compared with the oracle at that tolerance; its result must also meet
tol on the oracle's direct true residual.
Sizes span several CTAs / tiles and end in ragged tails (n not a multiple of
the 256-thread CTA or the 64-wide small-matrix tile).
"""
import numpy as np
import pytest

import paper_2605_28274_gb300 as ps
import workloads as wl
from oracle import exact, factorized as fz, residual

pytestmark = pytest.mark.gpu

TOL_X = 1e-10  # relative Frobenius error of X in FP64 mode
STOP_MARGIN = 0.4  # default sylv_options.stop_margin of a certified FP64 solve


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_solve(A, B, C1, C2, method, tol, maxit, lyapunov=False, precision="fp64", **kw):
    with ps.Solver(A, B, C1, C2, precision=precision, lyapunov=lyapunov, **kw) as sv:
        info = sv.cg(tol, maxit) if method == "cg" else sv.bicgstab(tol, maxit)
        V, Xh, W = sv.factors()
        hist = sv.history()
        H = sv.hessenberg(0)
    return info, V, Xh, W, hist, H


def oracle_solve(A, B, C1, C2, method, tol, maxit, lyapunov=False):
    As = A.to_scipy()
    Bs = None if lyapunov else B.to_scipy()
    if method == "cg":
        return fz.factorized_cg(As, Bs, C1, None if lyapunov else C2, tol, maxit, lyapunov=lyapunov)
    return fz.factorized_bicgstab(As, Bs, C1, C2, tol, maxit)


def ragged_spd(n, seed):
    return wl.random_sparse(n, 3, seed, spd=True)


def with_empty_rows(n, seed):
    """Random sparse matrix in which every 7th row is empty (ragged row lengths)."""
    A = wl.random_sparse(n, 4, seed)
    D = A.to_scipy().tolil()
    for i in range(0, n, 7):
        D.rows[i] = []
        D.data[i] = []
    M = D.tocsr()
    return wl.CSR(n, n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


# ------------------------------------------------------------------ sparse apply
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spmm_parity(k, precision):
    n, m = 1037, 515  # ragged: not multiples of the CTA size
    A, B = with_empty_rows(n, 1), with_empty_rows(m, 2)
    C1, C2 = wl.rhs(n, m, 2, 0)
    X = np.random.default_rng(k).standard_normal((n, k))
    Xb = np.random.default_rng(k + 1).standard_normal((m, k))
    with ps.Solver(A, B, C1, C2, precision=precision) as sv:
        Y = sv.apply(0, X)
        Yb = sv.apply(1, Xb)
    ref = A.to_scipy() @ X
    refb = B.to_scipy().T @ Xb
    tol = 1e-14 if precision == "fp64" else 2e-6
    assert rel(Y, ref) < tol
    assert rel(Yb, refb) < tol
    assert np.all(Y[::7] == 0.0)  # empty rows give exact zeros


# ------------------------------------------------------------------ factorized CG
def direct_rel(A, B, C1, C2, V, Xh, W):
    return residual.direct(A.to_scipy(), B.to_scipy(), C1, C2, V, Xh, W) / np.linalg.norm(C1 @ C2.T)


def test_cg_laplacian_400_matches_oracle_and_closed_form():
    # the printed stop test of Algorithm 4.1 (no certificate): same iterations as the oracle
    p = wl.cfg_laplace_cg(N=20, s=1)
    info, V, Xh, W, hist, H = gpu_solve(p.A, p.B, p.C1, p.C2, "cg", 1e-8, 200, no_true_residual=True)
    ref = oracle_solve(p.A, p.B, p.C1, p.C2, "cg", 1e-8, 200)
    assert info["status"] == ps.SYLV_OK and ref.status == "converged"
    assert info["iters"] == ref.iters
    assert info["width"] == ref.iters * 1
    np.testing.assert_allclose(hist, ref.history, rtol=1e-8, atol=0)
    X, Xo = V @ Xh @ W.T, ref.X()
    assert rel(X, Xo) < TOL_X
    Xs = exact.laplacian_exact(20, p.C1 @ p.C2.T)
    assert rel(X, Xs) < 357 * 1e-8  # kappa(F) times the residual tolerance
    Ho = ref.basisA.Hk(ref.iters + 1, ref.iters)
    assert rel(H, Ho) < 1e-12


def test_cg_laplacian_400_certified_stop_meets_tol():
    # the default solve: recurrence test at STOP_MARGIN * tol, then the float64 true-residual
    # certificate; the oracle's direct residual of the returned factors is below tol
    p = wl.cfg_laplace_cg(N=20, s=1)
    tol = 1e-8
    info, V, Xh, W, hist, H = gpu_solve(p.A, p.B, p.C1, p.C2, "cg", tol, 200)
    ref = oracle_solve(p.A, p.B, p.C1, p.C2, "cg", tol * STOP_MARGIN, 200)
    assert info["status"] == ps.SYLV_OK and ref.status == "converged"
    assert info["iters"] == ref.iters
    assert rel(V @ Xh @ W.T, ref.X()) < TOL_X
    assert 0 < info["true_rel_bound"] <= tol
    t = direct_rel(p.A, p.B, p.C1, p.C2, V, Xh, W)
    assert t <= tol and info["true_rel_res"] <= info["true_rel_bound"]


@pytest.mark.parametrize("s", [2, 3, 5])
def test_cg_sylvester_ragged_iterates(s):
    A = wl.laplacian_2d(23, 0.3)  # n = 529
    B = ragged_spd(300, 5)
    C1, C2 = wl.rhs(A.nrows, B.nrows, s, 3)
    for maxit in (1, 2, 7):  # iterate by iterate (ENOTCONV at maxit)
        info, V, Xh, W, hist, H = gpu_solve(A, B, C1, C2, "cg", 0.0, maxit)
        ref = oracle_solve(A, B, C1, C2, "cg", 0.0, maxit)
        assert info["status"] == ps.SYLV_ENOTCONV and info["iters"] == maxit
        assert rel(V @ Xh @ W.T, ref.X()) < TOL_X
    info, V, Xh, W, hist, H = gpu_solve(A, B, C1, C2, "cg", 1e-9, 300)
    ref = oracle_solve(A, B, C1, C2, "cg", 1e-9 * STOP_MARGIN, 300)
    assert info["status"] == ps.SYLV_OK and info["true_rel_bound"] <= 1e-9
    assert abs(info["iters"] - ref.iters) <= 1
    assert rel(V @ Xh @ W.T, ref.X()) < TOL_X * 10 if info["iters"] != ref.iters else rel(V @ Xh @ W.T, ref.X()) < TOL_X


def test_lyapunov_cg_symmetric_and_matches_oracle():
    A = wl.laplacian_2d(30, 0.25)  # n = 900
    C1, _ = wl.rhs(900, None, 2, 4)
    info, V, Xh, W, hist, H = gpu_solve(A, None, C1, None, "cg", 1e-10, 400, lyapunov=True)
    ref = oracle_solve(A, None, C1, None, "cg", 1e-10 * STOP_MARGIN, 400, lyapunov=True)
    assert info["status"] == ps.SYLV_OK and ref.status == "converged"
    assert info["iters"] == ref.iters
    assert np.array_equal(Xh, Xh.T)
    X = V @ Xh @ V.T
    assert np.linalg.norm(X - X.T) <= 1e-12 * np.linalg.norm(X)
    assert rel(X, ref.X()) < TOL_X
    assert np.array_equal(V, W)


# ------------------------------------------------------------------ factorized BiCGSTAB
@pytest.mark.parametrize("NA,NB,s", [(9, 7, 2), (10, 8, 5), (11, 5, 1)])
def test_bicgstab_convdiff_matches_oracle(NA, NB, s):
    A, B = wl.convdiff_3d(NA, 1), wl.convdiff_3d(NB, 2)
    C1, C2 = wl.rhs(A.nrows, B.nrows, s, 0)
    for maxit in (1, 3):
        info, V, Xh, W, hist, H = gpu_solve(A, B, C1, C2, "bicgstab", 0.0, maxit)
        ref = oracle_solve(A, B, C1, C2, "bicgstab", 0.0, maxit)
        assert info["iters"] == maxit and info["width"] == 2 * maxit * s
        assert rel(V @ Xh @ W.T, ref.X()) < TOL_X
        assert rel(H, ref.basisA.Hk(2 * maxit + 1, 2 * maxit)) < 1e-12
    info, V, Xh, W, hist, H = gpu_solve(A, B, C1, C2, "bicgstab", 1e-8, 300)
    ref = oracle_solve(A, B, C1, C2, "bicgstab", 1e-8 * STOP_MARGIN, 300)
    assert info["status"] == ps.SYLV_OK and ref.status == "converged"
    assert info["true_rel_bound"] <= 1e-8 and direct_rel(A, B, C1, C2, V, Xh, W) <= 1e-8
    assert abs(info["iters"] - ref.iters) <= max(2, ref.iters // 10)
    k = min(info["iters"], ref.iters, 10)
    np.testing.assert_allclose(hist[: k + 1], ref.history[: k + 1], rtol=1e-7)
    X = V @ Xh @ W.T
    Xe = exact.kron_solve(A.to_dense(), B.to_dense(), C1 @ C2.T) if A.nrows * B.nrows <= 60000 else ref.X()
    assert rel(X, ref.X()) < max(TOL_X, 10 * rel(ref.X(), Xe))


def test_exhausted_block_krylov_space_converges_to_exact():
    n, s = 12, 3
    A, B = ragged_spd(n, 41), ragged_spd(n, 42)
    C1, C2 = wl.rhs(n, n, s, 1)
    info, V, Xh, W, hist, H = gpu_solve(A, B, C1, C2, "bicgstab", 1e-12, 100)
    assert info["status"] == ps.SYLV_OK
    Xe = exact.kron_solve(A.to_dense(), B.to_dense(), C1 @ C2.T)
    assert rel(V @ Xh @ W.T, Xe) < 1e-9


# ------------------------------------------------------------------ edge cases
def test_edge_cases():
    A = wl.laplacian_2d(10)
    C1, C2 = wl.rhs(100, 100, 2, 0)
    with ps.Solver(A, A, C1, C2) as sv:
        info = sv.cg(1e-8, 0)
        assert info["status"] == ps.SYLV_ENOTCONV and info["width"] == 0
        info = sv.bicgstab(1e-8, 2)
        assert info["status"] == ps.SYLV_ENOTCONV and info["width"] == 8
        V, Xh, W = sv.factors()
        assert V.shape == (100, 8) and Xh.shape == (8, 8)
        assert np.allclose(V.T @ V, np.eye(8), atol=1e-13)
        # a second solve on the same handle reuses the device buffers
        info = sv.cg(1e-8, 200)
        assert info["status"] == ps.SYLV_OK
    # rank-deficient right-hand side factor: the thin QR of C1 breaks down
    with ps.Solver(A, A, np.zeros((100, 1)), np.ones((100, 1))) as sv:
        assert sv.cg(1e-8, 10)["status"] == ps.SYLV_EBREAKDOWN
    Cd = np.ones((100, 2))
    with ps.Solver(A, A, Cd, C2) as sv:
        assert sv.bicgstab(1e-8, 10)["status"] == ps.SYLV_EBREAKDOWN
    # non-finite input
    Cn = C1.copy()
    Cn[5, 1] = np.nan
    with pytest.raises(ps.SylvError) as e:
        ps.Solver(A, A, Cn, C2)
    assert e.value.code == ps.SYLV_ENONFINITE
    # CG on an indefinite operator breaks down (<P, Q> <= 0)
    Ai = wl.laplacian_2d(10, -6.0)
    with ps.Solver(Ai, Ai, C1, C2) as sv:
        info = sv.cg(1e-8, 100)
        assert info["status"] == ps.SYLV_EBREAKDOWN

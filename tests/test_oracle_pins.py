"""Pins of the CPU oracle against things other than itself.

Each test ties one oracle function to a closed form, a library routine used as
an independent reference (LAPACK Bartels-Stewart, a dense Kronecker solve),
an invariant the paper states, or brute force on tiny inputs.  A plausible
mistake anywhere in the oracle (a dropped term, a wrong sign or index, a
transposed operand, a wrong padding) makes at least one of them fail; the
last tests plant such mistakes in a copy of the operator and check that the
pins catch them.
"""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import exact, factorized as fz, matrix_oriented as mo, residual

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def small_spd(n, seed):
    return wl.random_sparse(n, 2, seed, spd=True).to_scipy()


# ---------------------------------------------------------------- exact solvers
def test_bartels_stewart_vs_kronecker():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((6, 6)) + 6 * np.eye(6)
    B = rng.standard_normal((4, 4)) + 6 * np.eye(4)
    C = rng.standard_normal((6, 4))
    X1 = exact.bartels_stewart(A, B, C)
    X2 = exact.kron_solve(A, B, C)
    assert rel(X1, X2) < 1e-13
    assert np.linalg.norm(A @ X1 + X1 @ B - C) < 1e-12 * np.linalg.norm(C)


def test_diagonal_closed_form():
    rng = np.random.default_rng(1)
    a, b = rng.random(7) + 0.5, rng.random(5) + 0.5
    C = rng.standard_normal((7, 5))
    assert rel(exact.diagonal_exact(a, b, C), exact.kron_solve(np.diag(a), np.diag(b), C)) < 1e-14


def test_laplacian_closed_form():
    N = 5
    L = wl.laplacian_2d(N).to_dense()
    C = np.random.default_rng(2).standard_normal((N * N, N * N))
    assert rel(exact.laplacian_exact(N, C), exact.kron_solve(L, L, C)) < 1e-12


# ---------------------------------------------------- matrix-oriented methods
def test_matrix_oriented_cg_converges_to_exact():
    A, B = small_spd(12, 1), small_spd(9, 2)
    C1, C2 = wl.rhs(12, 9, 2, 0)
    C = C1 @ C2.T
    r = mo.cg(A, B, C, 1e-12, 500)
    assert r.status == "converged"
    assert rel(r.X, exact.bartels_stewart(A.toarray(), B.toarray(), C)) < 1e-10


def test_matrix_oriented_first_iterate_brute_force():
    A, B = small_spd(8, 3), small_spd(6, 4)
    C = np.random.default_rng(3).standard_normal((8, 6))
    r = mo.cg(A, B, C, 0.0, 1, keep_iterates=True)
    AC = A.toarray() @ C + C @ B.toarray()
    alpha = np.sum(C * C) / np.sum(C * AC)  # X_1 = alpha_0 R_0 with R_0 = C
    assert rel(r.iterates[1], alpha * C) < 1e-14
    rb = mo.bicgstab(A, B, C, 0.0, 1, keep_iterates=True)
    al = np.sum(C * C) / np.sum(C * AC)
    S = C - al * AC
    T = A.toarray() @ S + S @ B.toarray()
    om = np.sum(T * S) / np.sum(T * T)
    assert rel(rb.iterates[1], al * C + om * S) < 1e-14


def test_matrix_oriented_bicgstab_converges_to_exact():
    A = wl.convdiff_3d(3, 1).to_scipy()
    B = wl.convdiff_3d(2, 2).to_scipy()
    C1, C2 = wl.rhs(27, 8, 2, 0)
    C = C1 @ C2.T
    r = mo.bicgstab(A, B, C, 1e-12, 300)
    assert r.status == "converged"
    assert rel(r.X, exact.kron_solve(A.toarray(), B.toarray(), C)) < 1e-9


# ------------------------------------------------------------- factor pieces
def test_thin_qr_properties():
    Y = np.random.default_rng(5).standard_normal((30, 4))
    Q, R = fz.thin_qr(Y)
    assert np.allclose(Q.T @ Q, np.eye(4), atol=1e-14)
    assert np.allclose(Q @ R, Y, atol=1e-13)
    assert np.allclose(R, np.triu(R)) and np.all(np.diag(R) > 0)


@pytest.mark.parametrize("kind", ["lanczos", "arnoldi"])
def test_block_krylov_relation_and_span(kind):
    n, s, k = 60, 3, 6
    A = small_spd(n, 7) if kind == "lanczos" else wl.convdiff_3d(4, 3).to_scipy()
    n = A.shape[0]
    C = np.random.default_rng(6).standard_normal((n, s))
    b = fz.BlockKrylovBasis(A, C, kind)
    for _ in range(k):
        b.step()
    Vk, Vk1 = b.V(k), b.V(k + 1)
    H = b.Hk(k + 1, k)
    # eq. (3.4): A V_k = V_{k+1} H_{k+1,k}
    assert np.linalg.norm(A @ Vk - Vk1 @ H) < 1e-12 * np.linalg.norm(A @ Vk)
    if kind == "arnoldi":
        assert np.allclose(Vk1.T @ Vk1, np.eye((k + 1) * s), atol=1e-13)
        assert np.allclose(np.tril(H, -s - 1), 0)  # block upper Hessenberg
    else:
        assert np.allclose(Vk1.T @ Vk1, np.eye((k + 1) * s), atol=1e-8)  # no reorthogonalisation
        for a in range(k + 1):  # block tridiagonal
            for c in range(k):
                if abs(a - c) > 1:
                    assert np.all(H[a * s:(a + 1) * s, c * s:(c + 1) * s] == 0)
    # span: K_{k+1}(A, C) = range(V_{k+1}) (Prop. 3.1 notation)
    K = [C]
    for _ in range(k):
        K.append(A @ K[-1])
    K = np.hstack(K)
    proj = Vk1 @ (Vk1.T @ K)
    assert np.linalg.norm(proj - K) < 1e-9 * np.linalg.norm(K)
    assert np.allclose(Vk1[:, :s] @ b.R0, C, atol=1e-12)


def test_block_krylov_exhaustion():
    n, s = 12, 3  # the space is exhausted after n/s = 4 blocks
    A = small_spd(n, 9)
    C = np.random.default_rng(8).standard_normal((n, s))
    b = fz.BlockKrylovBasis(A, C, "arnoldi")
    for _ in range(6):
        b.step()
    assert b.exhausted
    V = b.V(4)
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)
    assert np.all(b.blocks[4] == 0) and np.all(b.blocks[5] == 0)
    assert np.linalg.norm(A @ b.V(6) - b.V(7) @ b.Hk(7, 6)) < 1e-11


def random_basis_pair(n, m, s, k, seed):
    A = small_spd(n, seed)
    Bm = wl.convdiff_3d(3, seed).to_scipy()[:m, :m]
    C1, C2 = wl.rhs(n, m, s, seed)
    bA = fz.BlockKrylovBasis(A, C1, "arnoldi")
    bB = fz.BlockKrylovBasis(Bm.T, C2, "arnoldi")
    for _ in range(k):
        bA.step()
        bB.step()
    return A, Bm, bA, bB


def test_small_sylvester_operator_brute_force():
    """eq. (3.7): A(V_k Z W_k^T) + (V_k Z W_k^T) B = V_{k+1} S(Z) W_{k+1}^T."""
    s, k = 2, 4
    A, Bm, bA, bB = random_basis_pair(30, 27, s, k, 11)
    Z = np.random.default_rng(1).standard_normal((k * s, k * s))
    X = bA.V(k) @ Z @ bB.V(k).T
    lhs = A @ X + (Bm.T @ X.T).T
    Q = fz.small_sylvester(bA.Hk(k + 1, k), Z, bB.Hk(k + 1, k))
    assert Q.shape == ((k + 1) * s, (k + 1) * s)
    rhs = bA.V(k + 1) @ Q @ bB.V(k + 1).T
    assert rel(rhs, lhs) < 1e-12


def test_small_lyapunov_operator():
    s, k = 2, 3
    A = small_spd(20, 3)
    C = np.random.default_rng(0).standard_normal((20, s))
    b = fz.BlockKrylovBasis(A, C, "lanczos")
    for _ in range(k):
        b.step()
    Z = np.random.default_rng(2).standard_normal((k * s, k * s))
    Z = Z + Z.T
    H = b.Hk(k + 1, k)
    Q1 = fz.small_lyapunov(H, Z)
    assert np.array_equal(Q1, Q1.T)
    assert rel(Q1, fz.small_sylvester(H, Z, H)) < 1e-14
    X = b.V(k) @ Z @ b.V(k).T
    assert rel(b.V(k + 1) @ Q1 @ b.V(k + 1).T, A @ X + X @ A.T) < 1e-10


def test_inner_product_identity():
    """eq. (3.6): <V X W^T, V Y W^T> = <X, Y> for orthonormal V, W."""
    s, k = 2, 3
    _, _, bA, bB = random_basis_pair(25, 27, s, k, 4)
    rng = np.random.default_rng(3)
    X, Y = rng.standard_normal((2, k * s, k * s))
    big = np.sum((bA.V(k) @ X @ bB.V(k).T) * (bA.V(k) @ Y @ bB.V(k).T))
    assert abs(big - fz.inner(X, Y)) < 1e-12 * abs(big) + 1e-13


# ---------------------------------------- factorized == matrix-oriented (Sec. 5.1)
def test_factorized_cg_equals_matrix_oriented_iterates():
    A, B = small_spd(40, 21), small_spd(35, 22)
    C1, C2 = wl.rhs(40, 35, 2, 0)
    rf = fz.factorized_cg(A, B, C1, C2, 1e-10, 200, keep_iterates=True)
    rm = mo.cg(A, B, C1 @ C2.T, 1e-10, 200, keep_iterates=True)
    assert rf.status == rm.status == "converged"
    assert abs(rf.iters - rm.iters) <= 2
    for k in range(1, min(20, rf.iters) + 1):
        assert rel(rf.X_at(k, k), rm.iterates[k]) < 1e-10, k
        assert abs(rf.history[k] - rm.history[k]) <= 1e-9 * rm.history[k] + 1e-15
    # rank(X_k) <= k s (Corollary 3.2)
    for k in (1, 2, 3):
        assert np.linalg.matrix_rank(rm.iterates[k], tol=1e-10 * np.linalg.norm(rm.iterates[k])) <= k * 2


def test_factorized_bicgstab_equals_matrix_oriented_iterates():
    A = wl.convdiff_3d(5, 1).to_scipy()
    B = wl.convdiff_3d(4, 2).to_scipy()
    C1, C2 = wl.rhs(125, 64, 2, 0)
    rf = fz.factorized_bicgstab(A, B, C1, C2, 1e-10, 200, keep_iterates=True)
    rm = mo.bicgstab(A, B, C1 @ C2.T, 1e-10, 200, keep_iterates=True)
    assert rf.status == rm.status == "converged"
    assert abs(rf.iters - rm.iters) <= max(2, rm.iters // 10)
    for k in range(1, min(12, rf.iters) + 1):
        assert rel(rf.X_at(k, 2 * k), rm.iterates[k]) < 1e-10, k
        assert rank_at_most(rm.iterates[k], 2 * k * 2)
    X = exact.kron_solve(A.toarray(), B.toarray(), C1 @ C2.T)
    assert rel(rf.X(), X) < 1e-8


def rank_at_most(X, r):
    return np.linalg.matrix_rank(X, tol=1e-10 * np.linalg.norm(X)) <= r


def test_lyapunov_variant_symmetric_and_equal_to_sylvester():
    A = small_spd(30, 31)
    C1, _ = wl.rhs(30, None, 2, 0)
    ry = fz.factorized_cg(A, None, C1, None, 1e-10, 200, lyapunov=True, keep_iterates=True)
    rs = fz.factorized_cg(A, A, C1, C1, 1e-10, 200, keep_iterates=True)
    assert ry.status == rs.status == "converged"
    assert np.array_equal(ry.Xhat, ry.Xhat.T)
    X = ry.X()
    assert np.linalg.norm(X - X.T) <= 1e-12 * np.linalg.norm(X)
    for k in range(1, 15):
        assert rel(ry.X_at(k, k), rs.X_at(k, k)) < 1e-10
    Xe = exact.bartels_stewart(A.toarray(), A.toarray(), C1 @ C1.T)
    assert rel(X, Xe) < 1e-8


def test_laplacian_workload_against_closed_form():
    p = wl.cfg_laplace_cg(N=20, s=1)
    r = fz.factorized_cg(p.A.to_scipy(), p.B.to_scipy(), p.C1, p.C2, 1e-12, 400)
    assert r.status == "converged"
    X = exact.laplacian_exact(20, p.C1 @ p.C2.T)
    assert rel(r.X(), X) < 1e-9  # kappa(F) = 357 times the 1e-12 residual


def test_diagonal_case_closed_form():
    rng = np.random.default_rng(12)
    a, b = rng.random(300) + 1.0, rng.random(200) + 1.0
    A, B = wl.diagonal(a).to_scipy(), wl.diagonal(b).to_scipy()
    C1, C2 = wl.rhs(300, 200, 2, 0)
    r = fz.factorized_cg(A, B, C1, C2, 1e-12, 300)
    assert r.status == "converged"
    assert rel(r.X(), exact.diagonal_exact(a, b, C1 @ C2.T)) < 1e-11
    r2 = fz.factorized_bicgstab(A, B, C1, C2, 1e-12, 300)
    assert r2.status == "converged"
    assert rel(r2.X(), exact.diagonal_exact(a, b, C1 @ C2.T)) < 1e-10


def test_exhausted_spaces_reach_exact_solution():
    n, s = 12, 3  # both block Krylov spaces fill up after 4 steps
    A, B = small_spd(n, 41), small_spd(n, 42)
    C1, C2 = wl.rhs(n, n, s, 1)
    r = fz.factorized_bicgstab(A, B, C1, C2, 1e-12, 100)
    assert r.status == "converged" and r.basisA.exhausted and r.basisB.exhausted
    assert rel(r.X(), exact.kron_solve(A.toarray(), B.toarray(), C1 @ C2.T)) < 1e-9


# ------------------------------------------------------------ true residual
def test_true_residual_factored_equals_direct():
    A = wl.convdiff_3d(5, 1).to_scipy()
    B = wl.convdiff_3d(4, 2).to_scipy()
    C1, C2 = wl.rhs(125, 64, 2, 0)
    r = fz.factorized_bicgstab(A, B, C1, C2, 1e-9, 200)
    d = residual.direct(A, B, C1, C2, r.V, r.Xhat, r.W)
    f = residual.factored(A, B, C1, C2, r.V, r.Xhat, r.W)
    c = residual.rhs_norm(C1, C2)
    assert abs(c - np.linalg.norm(C1 @ C2.T)) < 1e-13 * c
    assert abs(d - f) < 1e-12 * c
    assert abs(d / c - r.history[-1]) < 1e-9  # monitored == true with orthonormal bases
    assert d / c <= 1e-9 * 1.01


# ------------------------------------------------------- paper's printed counts
def test_paper_table1_iteration_counts_soft():
    """Table 1: factorized CG on the 100 x 100 Laplacian Lyapunov equation, tol 1e-6."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "paper_table1_cg_iterations.txt"))
            if ln.strip() and not ln.startswith("#")]
    L = wl.laplacian_2d(100).to_scipy()
    for s, its in [(int(a), int(b)) for a, b in rows][:2]:
        C1, _ = wl.rhs(10000, None, s, 0)
        r = fz.factorized_cg(L, None, C1, None, 1e-6, 400, lyapunov=True)
        assert r.status == "converged"
        assert abs(r.iters - its) <= 0.03 * its, (s, r.iters, its)


# ----------------------------------------- planted mistakes are caught (mutation)
def test_planted_mistakes_fail_the_pins():
    s, k = 2, 4
    A, Bm, bA, bB = random_basis_pair(30, 27, s, k, 11)
    Z = np.random.default_rng(1).standard_normal((k * s, k * s))
    X = bA.V(k) @ Z @ bB.V(k).T
    lhs = A @ X + (Bm.T @ X.T).T
    H, G = bA.Hk(k + 1, k), bB.Hk(k + 1, k)
    r = k * s

    def transposed_operand(H, Z, G):  # Z^T G^T instead of Z G^T
        out = np.zeros((r + s, r + s))
        out[:, :r] += H @ Z
        out[:r, :] += Z.T @ G.T
        return out

    def wrong_sign(H, Z, G):
        out = np.zeros((r + s, r + s))
        out[:, :r] += H @ Z
        out[:r, :] -= Z @ G.T
        return out

    def dropped_term(H, Z, G):
        out = np.zeros((r + s, r + s))
        out[:, :r] += H @ Z
        return out

    def wrong_pad(H, Z, G):  # Z G^T placed in the bottom rows instead of the top
        out = np.zeros((r + s, r + s))
        out[:, :r] += H @ Z
        out[s:, :] += Z @ G.T
        return out

    for bad in (transposed_operand, wrong_sign, dropped_term, wrong_pad):
        Q = bad(H, Z, G)
        assert rel(bA.V(k + 1) @ Q @ bB.V(k + 1).T, lhs) > 1e-3, bad.__name__


# ------------------------------------------- CGS (Sec. 4 names it; Sonneveld 1989)
def kron_operator(A, B):
    """F = I (x) A + B^T (x) I, so that F vec(X) = vec(A X + X B) (eq. 1.2, column-major vec)."""
    import scipy.sparse as sp

    n, m = A.shape[0], B.shape[0]
    return (sp.kron(sp.eye(m), A) + sp.kron(B.T, sp.eye(n))).tocsr()


def test_matrix_oriented_cgs_matches_scipy_cgs_on_kronecker_system():
    import scipy.sparse.linalg as spla

    A = wl.convdiff_3d(5, 1).to_scipy()
    B = wl.convdiff_3d(4, 2).to_scipy()
    C1, C2 = wl.rhs(125, 64, 2, 0)
    C = C1 @ C2.T
    rm = mo.cgs(A, B, C, 0.0, 10, keep_iterates=True)
    xs = []
    spla.cgs(kron_operator(A, B), C.flatten(order="F"), rtol=0.0, atol=0.0, maxiter=10,
             callback=lambda x: xs.append(x.copy()))
    assert len(xs) == 10
    for k in range(1, 11):
        assert rel(rm.iterates[k].flatten(order="F"), xs[k - 1]) < 1e-12, k


def test_matrix_oriented_cgs_converges_to_exact():
    A = wl.convdiff_3d(5, 1).to_scipy()
    B = wl.convdiff_3d(4, 2).to_scipy()
    C1, C2 = wl.rhs(125, 64, 2, 0)
    r = mo.cgs(A, B, C1 @ C2.T, 1e-12, 200)
    assert r.status == "converged"
    X = exact.bartels_stewart(A.toarray(), B.toarray(), C1 @ C2.T)
    assert rel(r.X, X) < 1e-9


def test_factorized_cgs_equals_matrix_oriented_iterates():
    A = wl.convdiff_3d(5, 1).to_scipy()
    B = wl.convdiff_3d(4, 2).to_scipy()
    C1, C2 = wl.rhs(125, 64, 2, 0)
    rf = fz.factorized_cgs(A, B, C1, C2, 1e-10, 200, keep_iterates=True)
    rm = mo.cgs(A, B, C1 @ C2.T, 1e-10, 200, keep_iterates=True)
    assert rf.status == rm.status == "converged"
    assert abs(rf.iters - rm.iters) <= max(2, rm.iters // 10)
    for k in range(1, min(12, rf.iters) + 1):
        assert rf.Xhats[k].shape[0] == (2 * k) * 2
        assert rel(rf.X_at(k, 2 * k), rm.iterates[k]) < 1e-10, k
        assert rank_at_most(rm.iterates[k], 2 * k * 2)
    np.testing.assert_allclose(rf.history[:12], rm.history[:12], rtol=1e-8)
    X = exact.kron_solve(A.toarray(), B.toarray(), C1 @ C2.T)
    assert rel(rf.X(), X) < 1e-8


def test_factorized_cgs_diagonal_case_closed_form():
    rng = np.random.default_rng(9)
    a = rng.uniform(1.0, 3.0, 40)
    b = rng.uniform(1.0, 3.0, 30)
    A = wl.diagonal(a).to_scipy()
    B = wl.diagonal(b).to_scipy()
    C1, C2 = wl.rhs(40, 30, 2, 3)
    r = fz.factorized_cgs(A, B, C1, C2, 1e-11, 60)
    assert r.status == "converged"
    assert rel(r.X(), exact.diagonal_exact(a, b, C1 @ C2.T)) < 1e-9


def test_planted_cgs_mistake_fails_the_scipy_pin():
    """A CGS recurrence with beta instead of beta^2 in the P update drifts away from the
    library's CGS iterates: the scipy pin would catch that mistake in the oracle."""
    import scipy.sparse.linalg as spla

    A = wl.convdiff_3d(5, 1).to_scipy()
    B = wl.convdiff_3d(4, 2).to_scipy()
    C1, C2 = wl.rhs(125, 64, 2, 0)
    C = C1 @ C2.T
    X = np.zeros_like(C)
    R = C.copy()
    Rt, U, P = R.copy(), R.copy(), R.copy()
    rho = mo.inner(Rt, R)
    its = []
    for _ in range(6):
        V = mo.sylvester_op(A, B, P)
        alpha = rho / mo.inner(Rt, V)
        Q = U - alpha * V
        X = X + alpha * (U + Q)
        R = R - alpha * mo.sylvester_op(A, B, U + Q)
        its.append(X.copy())
        rho_new = mo.inner(Rt, R)
        beta = rho_new / rho
        rho = rho_new
        U = R + beta * Q
        P = U + beta * (Q + P)  # planted: beta instead of beta^2 on P_k
    xs = []
    spla.cgs(kron_operator(A, B), C.flatten(order="F"), rtol=0.0, atol=0.0, maxiter=6,
             callback=lambda x: xs.append(x.copy()))
    assert max(rel(its[k].flatten(order="F"), xs[k]) for k in range(6)) > 1e-3


# ---------------------------------------------- CR (Sec. 4 names it; Stiefel 1955)
def spd_pair():
    return wl.laplacian_2d(9).to_scipy(), wl.laplacian_2d(7).to_scipy()


def test_matrix_oriented_cr_matches_scipy_minres_on_kronecker_system():
    """For a self-adjoint operator CR and MINRES both minimise ||R|| over the same Krylov
    space, so their iterates coincide; scipy's MINRES is the independent reference."""
    import scipy.sparse.linalg as spla

    A, B = spd_pair()
    C1, C2 = wl.rhs(81, 49, 2, 0)
    C = C1 @ C2.T
    rm = mo.cr(A, B, C, 0.0, 12, keep_iterates=True)
    xs = []
    spla.minres(kron_operator(A, B), C.flatten(order="F"), rtol=1e-300, maxiter=12,
                callback=lambda x: xs.append(x.copy()))
    assert len(xs) == 12
    for k in range(1, 13):
        assert rel(rm.iterates[k].flatten(order="F"), xs[k - 1]) < 1e-12, k


def test_factorized_cr_equals_matrix_oriented_iterates():
    A, B = spd_pair()
    C1, C2 = wl.rhs(81, 49, 2, 0)
    rf = fz.factorized_cr(A, B, C1, C2, 1e-10, 200, keep_iterates=True)
    rm = mo.cr(A, B, C1 @ C2.T, 1e-10, 200, keep_iterates=True)
    assert rf.status == rm.status == "converged"
    assert abs(rf.iters - rm.iters) <= 2
    for k in range(1, min(15, rf.iters) + 1):
        assert rf.Xhats[k].shape[0] == k * 2
        assert rel(rf.X_at(k, k), rm.iterates[k]) < 1e-10, k
        assert rank_at_most(rm.iterates[k], k * 2)
    np.testing.assert_allclose(rf.history[:15], rm.history[:15], rtol=1e-8)
    X = exact.bartels_stewart(A.toarray(), B.toarray(), C1 @ C2.T)
    assert rel(rf.X(), X) < 1e-8


def test_factorized_cr_lyapunov_symmetric_and_exact():
    A = wl.laplacian_2d(9, 0.5).to_scipy()
    C1, _ = wl.rhs(81, None, 3, 2)
    r = fz.factorized_cr(A, None, C1, None, 1e-11, 200, lyapunov=True)
    assert r.status == "converged"
    assert np.abs(r.Xhat - r.Xhat.T).max() == 0.0
    X = exact.bartels_stewart(A.toarray(), A.toarray(), C1 @ C1.T)
    assert rel(r.X(), X) < 1e-8
    r2 = fz.factorized_cr(A, A, C1, C1, 1e-11, 200)
    assert rel(r.X(), r2.X()) < 1e-9


def test_factorized_cr_diagonal_case_closed_form():
    rng = np.random.default_rng(10)
    a, b = rng.uniform(1.0, 3.0, 40), rng.uniform(1.0, 3.0, 30)
    A, B = wl.diagonal(a).to_scipy(), wl.diagonal(b).to_scipy()
    C1, C2 = wl.rhs(40, 30, 2, 3)
    r = fz.factorized_cr(A, B, C1, C2, 1e-11, 60)
    assert r.status == "converged"
    assert rel(r.X(), exact.diagonal_exact(a, b, C1 @ C2.T)) < 1e-9


def test_planted_cr_mistake_fails_the_minres_pin():
    """CR that forgets the beta L(P_k) term of the L(P) recurrence leaves MINRES's iterates."""
    import scipy.sparse.linalg as spla

    A, B = spd_pair()
    C1, C2 = wl.rhs(81, 49, 2, 0)
    C = C1 @ C2.T
    X = np.zeros_like(C)
    R = C.copy()
    LR = mo.sylvester_op(A, B, R)
    P, LP = R.copy(), LR.copy()
    rho = mo.inner(R, LR)
    its = []
    for _ in range(6):
        alpha = rho / mo.inner(LP, LP)
        X = X + alpha * P
        R = R - alpha * LP
        its.append(X.copy())
        LR = mo.sylvester_op(A, B, R)
        rho_new = mo.inner(R, LR)
        beta = rho_new / rho
        rho = rho_new
        P = R + beta * P
        LP = LR  # planted: dropped beta L(P_k)
    xs = []
    spla.minres(kron_operator(A, B), C.flatten(order="F"), rtol=1e-300, maxiter=6,
                callback=lambda x: xs.append(x.copy()))
    assert max(rel(its[k].flatten(order="F"), xs[k]) for k in range(6)) > 1e-3


# -------------------------------------------- GPBiCG (Sec. 4 names it; Zhang 1997)
def cd_pair():
    A = wl.convdiff_3d(5, 1).to_scipy()
    B = wl.convdiff_3d(4, 2).to_scipy()
    C1, C2 = wl.rhs(125, 64, 2, 0)
    return A, B, C1, C2


def test_gpbicg_with_eta_zero_is_bicgstab():
    """With eta = 0 in every step the GPBiCG recurrence is BiCGSTAB's (omega = zeta), itself
    pinned above: this ties every term except the eta terms."""
    A, B, C1, C2 = cd_pair()
    g = mo.gpbicg(A, B, C1 @ C2.T, 1e-10, 200, keep_iterates=True, eta_zero=True)
    b = mo.bicgstab(A, B, C1 @ C2.T, 1e-10, 200, keep_iterates=True)
    assert g.iters == b.iters
    for k in range(1, g.iters + 1):
        assert rel(g.iterates[k], b.iterates[k]) < 1e-12, k


def test_gpbicg_residual_is_orthogonal_to_LT_and_Y():
    """zeta, eta minimise ||T - zeta L(T) - eta Y||: the new residual is orthogonal to both."""
    A, B, C1, C2 = cd_pair()
    rec = []
    r = mo.gpbicg(A, B, C1 @ C2.T, 1e-10, 200, record=rec)
    assert r.status == "converged" and len(rec) >= 5
    for R, LT, Y in rec[1:]:
        assert abs(mo.inner(R, LT)) <= 1e-12 * np.linalg.norm(R) * np.linalg.norm(LT)
        assert abs(mo.inner(R, Y)) <= 1e-12 * np.linalg.norm(R) * np.linalg.norm(Y)


def test_matrix_oriented_gpbicg_converges_to_exact():
    A, B, C1, C2 = cd_pair()
    r = mo.gpbicg(A, B, C1 @ C2.T, 1e-12, 200)
    assert r.status == "converged"
    assert rel(r.X, exact.bartels_stewart(A.toarray(), B.toarray(), C1 @ C2.T)) < 1e-9


def test_factorized_gpbicg_equals_matrix_oriented_iterates():
    A, B, C1, C2 = cd_pair()
    rf = fz.factorized_gpbicg(A, B, C1, C2, 1e-10, 200, keep_iterates=True)
    rm = mo.gpbicg(A, B, C1 @ C2.T, 1e-10, 200, keep_iterates=True)
    assert rf.status == rm.status == "converged"
    assert abs(rf.iters - rm.iters) <= 1
    for k in range(1, min(12, rf.iters) + 1):
        assert rf.Xhats[k].shape[0] == (2 * k) * 2
        assert rel(rf.X_at(k, 2 * k), rm.iterates[k]) < 1e-10, k
        assert rank_at_most(rm.iterates[k], 2 * k * 2)
    np.testing.assert_allclose(rf.history[:12], rm.history[:12], rtol=1e-8)
    assert rel(rf.X(), exact.kron_solve(A.toarray(), B.toarray(), C1 @ C2.T)) < 1e-8


def test_factorized_gpbicg_diagonal_case_closed_form():
    rng = np.random.default_rng(11)
    a, b = rng.uniform(1.0, 3.0, 40), rng.uniform(1.0, 3.0, 30)
    A, B = wl.diagonal(a).to_scipy(), wl.diagonal(b).to_scipy()
    C1, C2 = wl.rhs(40, 30, 2, 3)
    r = fz.factorized_gpbicg(A, B, C1, C2, 1e-11, 60)
    assert r.status == "converged"
    assert rel(r.X(), exact.diagonal_exact(a, b, C1 @ C2.T)) < 1e-9


def test_planted_gpbicg_mistake_fails_the_orthogonality_pin():
    """A zeta with two inner products swapped no longer solves the 2 x 2 least-squares
    problem: the residual loses its orthogonality to L(T)."""
    A, B, C1, C2 = cd_pair()
    C = C1 @ C2.T
    R = C.copy()
    Rt, P, U, W, Z, Tp = R.copy(), 0 * R, 0 * R, 0 * R, 0 * R, 0 * R
    beta, rho = 0.0, mo.inner(R, R)
    worst = 0.0
    for k in range(6):
        P = R + beta * (P - U)
        LP = mo.sylvester_op(A, B, P)
        alpha = rho / mo.inner(Rt, LP)
        Y = Tp - R - alpha * W + alpha * LP
        T = R - alpha * LP
        LT = mo.sylvester_op(A, B, T)
        if k == 0:
            zeta, eta = mo.inner(LT, T) / mo.inner(LT, LT), 0.0
        else:
            yy, tt_, yt, ty, aa = mo.inner(Y, Y), mo.inner(LT, T), mo.inner(Y, T), mo.inner(LT, Y), mo.inner(LT, LT)
            den = aa * yy - ty * ty
            zeta = (yy * tt_ - ty * yt * 0.5) / den  # planted: a wrong term in zeta
            eta = (aa * yt - ty * tt_) / den
        U = zeta * LP + eta * (Tp - R + beta * U)
        Z = zeta * R + eta * Z - alpha * U
        R = T - eta * Y - zeta * LT
        if k > 0:
            worst = max(worst, abs(mo.inner(R, LT)) / (np.linalg.norm(R) * np.linalg.norm(LT)))
        rho_new = mo.inner(Rt, R)
        beta = (alpha / zeta) * (rho_new / rho)
        rho = rho_new
        W = LT + beta * LP
        Tp = T
    assert worst > 1e-6


# ------------------------------------------------- partial loss of rank (deflation)
def rank_losing_problem():
    """C1 = [c, A c, x]: the second basis block contains A c, already in the first block's span,
    so one column of every later block is (exactly, up to rounding) dependent."""
    A = wl.convdiff_3d(6, 1).to_scipy()
    B = wl.convdiff_3d(5, 2).to_scipy()
    rng = np.random.default_rng(3)
    c = rng.standard_normal(A.shape[0])
    C1 = np.column_stack([c, A @ c, rng.standard_normal(A.shape[0])])
    C2 = rng.standard_normal((B.shape[0], 3))
    return A, B, C1, C2


def test_partial_rank_loss_deflates_to_zero_columns():
    A, B, C1, C2 = rank_losing_problem()
    r = fz.factorized_bicgstab(A, B, C1, C2, 1e-10, 300)
    assert r.status == "converged" and r.basisA.deflated > 0
    V = r.basisA.V()
    norms = np.linalg.norm(V, axis=0)
    zero = norms == 0.0
    assert zero.sum() == r.basisA.deflated and not zero[:3].any()
    Vk = V[:, ~zero]
    assert np.abs(Vk.T @ Vk - np.eye(Vk.shape[1])).max() < 1e-12  # the kept columns stay orthonormal
    k = V.shape[1] - 3
    assert np.abs(A @ V[:, :k] - V @ r.basisA.H[: V.shape[1], :k]).max() < 1e-12  # eq. 3.4 still holds
    assert rel(r.X(), exact.bartels_stewart(A.toarray(), B.toarray(), C1 @ C2.T)) < 1e-8


@pytest.mark.parametrize("method", ["cgs", "gpbicg"])
def test_partial_rank_loss_other_arnoldi_methods(method):
    A, B, C1, C2 = rank_losing_problem()
    r = getattr(fz, "factorized_" + method)(A, B, C1, C2, 1e-10, 300)
    assert r.status == "converged" and r.basisA.deflated > 0
    assert rel(r.X(), exact.bartels_stewart(A.toarray(), B.toarray(), C1 @ C2.T)) < 1e-8


def test_partial_rank_loss_lanczos_methods():
    A, B = wl.laplacian_2d(8).to_scipy(), wl.laplacian_2d(7).to_scipy()
    rng = np.random.default_rng(4)
    c = rng.standard_normal(64)
    C1, C2 = np.column_stack([c, A @ c]), rng.standard_normal((49, 2))
    X = exact.bartels_stewart(A.toarray(), B.toarray(), C1 @ C2.T)
    for f in (fz.factorized_cg, fz.factorized_cr):
        r = f(A, B, C1, C2, 1e-10, 300)
        assert r.status == "converged" and r.basisA.deflated > 0
        assert rel(r.X(), X) < 1e-8


# ------------------------------------------------ final low-rank compression of X
def test_compression_is_the_best_low_rank_approximation():
    """Eckart-Young on a formed X: the compressed factors reproduce numpy's truncated SVD of X,
    and ||X - X_q||_F equals the discarded singular values' norm, within tol * ||X||_F."""
    from oracle import compress

    A = wl.convdiff_3d(6, 1).to_scipy()
    B = wl.convdiff_3d(5, 2).to_scipy()
    C1, C2 = wl.rhs(216, 125, 2, 0)
    r = fz.factorized_bicgstab(A, B, C1, C2, 1e-10, 300)
    X = r.X()
    for tol in (1e-2, 1e-5, 1e-9):
        Vq, sq, Wq = compress.compress(r.V, r.Xhat, r.W, tol)
        Xq = (Vq * sq) @ Wq.T
        sx = np.linalg.svd(X, compute_uv=False)
        q = compress.truncation_rank(sx, tol)
        assert len(sq) == q
        np.testing.assert_allclose(sq, sx[:q], rtol=1e-9, atol=1e-12 * sx[0])
        err = np.linalg.norm(X - Xq)
        assert abs(err - np.sqrt(np.sum(sx[q:] ** 2))) <= 1e-9 * np.linalg.norm(X)
        assert err <= tol * np.linalg.norm(X) * (1 + 1e-9)
        assert np.abs(Vq.T @ Vq - np.eye(q)).max() < 1e-12  # orthonormal compressed factors


def test_truncation_rank_rule():
    from oracle import compress

    sv = np.array([4.0, 3.0, 0.0])
    assert compress.truncation_rank(sv, 0.0) == 2
    assert compress.truncation_rank(sv, 0.6) == 1  # ||(3, 0)|| = 3 <= 0.6 * 5
    assert compress.truncation_rank(sv, 0.59) == 2
    assert compress.truncation_rank(sv, 1.0) == 0

"""Pins of the seeded input generators (nnz formulas, symmetry, M-matrix, spectrum)."""
import numpy as np
import pytest

import workloads as wl


@pytest.mark.parametrize("N", [1, 2, 5, 20])
def test_laplacian_nnz_and_symmetry(N):
    L = wl.laplacian_2d(N)
    assert L.nnz == 5 * N * N - 4 * N
    D = L.to_dense()
    assert np.array_equal(D, D.T)
    assert np.all(np.diag(D) == 4.0)


def test_laplacian_spectrum_closed_form():
    N = 7
    D = wl.laplacian_2d(N).to_dense()
    ev = np.sort(np.linalg.eigvalsh(D))
    p = np.arange(1, N + 1)
    lam1 = 2 - 2 * np.cos(p * np.pi / (N + 1))
    ref = np.sort((lam1[:, None] + lam1[None, :]).ravel())
    assert np.allclose(ev, ref, atol=1e-12)


@pytest.mark.parametrize("N,seed", [(3, 1), (6, 2), (9, 7)])
def test_convdiff_structure(N, seed):
    A = wl.convdiff_3d(N, seed)
    assert A.nnz == 7 * N**3 - 6 * N**2
    D = A.to_dense()
    off = D - np.diag(np.diag(D))
    assert np.all(np.diag(D) > 0) and np.all(off <= 0)
    rows = D.sum(axis=1)
    assert np.all(rows >= -1e-14) and np.any(rows > 1e-3)  # diagonally dominant M-matrix
    assert not np.allclose(D, D.T)  # convection makes it nonsymmetric
    w = wl.wind_direction(seed)
    assert abs(np.linalg.norm(w) - 1) < 1e-15
    h = 1.0 / (N + 1)
    assert np.isclose(D[0, 0], 6 + h * 10 * np.abs(w).sum())


def test_convdiff_workload_sizes():
    A = wl.convdiff_3d(64, 1)
    assert A.nrows == 262144 and A.nnz == 1810432
    B = wl.convdiff_3d(48, 2)
    assert B.nrows == 110592 and B.nnz == 760320


def test_transpose_and_rhs():
    A = wl.random_sparse(50, 3, 0)
    assert np.array_equal(A.transpose().to_dense(), A.to_dense().T)
    C1, C2 = wl.rhs(10, 7, 3, 0)
    D1, D2 = wl.rhs(10, 7, 3, 0)
    assert C1.shape == (10, 3) and C2.shape == (7, 3)
    assert np.array_equal(C1, D1) and np.array_equal(C2, D2)
    E1, E2 = wl.rhs(10, None, 3, 0)
    assert np.array_equal(E1, E2)


def test_batched_lyapunov_workload_draws():
    probs = wl.cfg_batched_lyapunov(count=64)
    assert len(probs) == 64
    for p in probs:
        N = p.meta["N"]
        assert 64 <= N <= 256 and p.s in (1, 2, 4) and 0 <= p.meta["sigma"] < 1
        assert p.A.nrows == N * N and p.C1.shape == (N * N, p.s) and p.lyapunov
    again = wl.cfg_batched_lyapunov(count=3)
    assert [q.meta["N"] for q in again] == [q.meta["N"] for q in probs[:3]]


def test_random_sparse_spd():
    A = wl.random_sparse(40, 3, 5, spd=True).to_dense()
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0

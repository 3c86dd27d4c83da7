"""Exact solutions of A X + X B = C used to pin the iterative oracles.

Test infrastructure only (see ``oracle/__init__``).

* ``bartels_stewart``: the dense Schur-based direct method the paper names for
  small sizes (Sec. 1), via LAPACK (``scipy.linalg.solve_sylvester``).
* ``kron_solve``: the vectorised system (I_m (x) A + B^T (x) I_n) vec(X) =
  vec(C) of eq. (1.2), solved densely (tiny sizes only).
* ``diagonal_exact``: A = diag(a), B = diag(b): X_ij = C_ij / (a_i + b_j).
* ``laplacian_exact``: A = B = the N x N 5-point Laplacian, whose eigenvectors
  are products of discrete sines: X = U ((U^T C U) ./ (lam_i + lam_j)) U^T.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def bartels_stewart(A: np.ndarray, B: np.ndarray, C: np.ndarray) -> np.ndarray:
    return scipy.linalg.solve_sylvester(np.asarray(A), np.asarray(B), np.asarray(C))


def kron_solve(A: np.ndarray, B: np.ndarray, C: np.ndarray) -> np.ndarray:
    n, m = C.shape
    F = np.kron(np.eye(m), A) + np.kron(B.T, np.eye(n))
    x = np.linalg.solve(F, C.reshape(-1, order="F"))
    return x.reshape((n, m), order="F")


def diagonal_exact(a: np.ndarray, b: np.ndarray, C: np.ndarray) -> np.ndarray:
    return C / (a[:, None] + b[None, :])


def laplacian_1d_sines(N: int):
    """Eigenpairs of tridiag(-1, 2, -1) of order N: S[i,p] = sqrt(2/(N+1)) sin((i+1)(p+1) pi/(N+1))."""
    i = np.arange(1, N + 1)
    S = np.sqrt(2.0 / (N + 1)) * np.sin(np.outer(i, i) * np.pi / (N + 1))
    lam = 2.0 - 2.0 * np.cos(i * np.pi / (N + 1))
    return S, lam


def laplacian_2d_eig(N: int):
    """Eigenpairs of the 5-point Laplacian with index i + N j: U = S (x) S, lam_pq = lam_p + lam_q."""
    S, lam = laplacian_1d_sines(N)
    U = np.kron(S, S)
    L = (lam[None, :] + lam[:, None]).reshape(-1)  # index p + N q <-> kron(S,S) column q*N + p
    return U, L


def laplacian_exact(N: int, C: np.ndarray) -> np.ndarray:
    """Solution of L X + X L = C for the N x N 5-point Laplacian L (diag 4, neighbours -1)."""
    U, lam = laplacian_2d_eig(N)
    Ct = U.T @ C @ U
    return U @ (Ct / (lam[:, None] + lam[None, :])) @ U.T

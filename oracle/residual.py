"""True residual ||C1 C2^T - A X - X B||_F of a factored iterate X = V X^ W^T.

Test infrastructure only (see ``oracle/__init__``).  The convergence test of
Algorithms 4.1/4.2 monitors ||R^_k|| (equal to the true residual only while V
and W stay orthonormal, eq. 3.6); these functions compute the true value.

* ``direct``: forms X and the residual (n m small).
* ``factored``: C1 C2^T - (A V) X^ W^T - V X^ (B^T W)^T = L M Rf^T with
  L = [C1, A V, V], Rf = [C2, W, B^T W] and M = blkdiag(I_s, -X^, -X^);
  Householder QR of L and Rf (L = Q_L T_L, Rf = Q_R T_R) gives
  ||residual||_F = ||T_L M T_R^T||_F without forming n x m matrices.
"""
from __future__ import annotations

import numpy as np


def direct(A, B, C1, C2, V, Xh, W) -> float:
    X = V @ Xh @ W.T
    R = C1 @ C2.T - np.asarray(A @ X) - np.asarray((B.T @ X.T).T)
    return float(np.linalg.norm(R))


def factored(A, B, C1, C2, V, Xh, W) -> float:
    s = C1.shape[1]
    r = Xh.shape[0]
    AV = np.asarray(A @ V)
    BtW = np.asarray(B.T @ W)
    L = np.hstack([C1, AV, V])
    Rf = np.hstack([C2, W, BtW])
    M = np.zeros((s + 2 * r, s + 2 * r))
    M[:s, :s] = np.eye(s)
    M[s:s + r, s:s + r] = -Xh
    M[s + r:, s + r:] = -Xh
    TL = np.linalg.qr(L, mode="r")
    TR = np.linalg.qr(Rf, mode="r")
    return float(np.linalg.norm(TL @ M @ TR.T))


def rhs_norm(C1, C2) -> float:
    """||C1 C2^T||_F = ||R1 R2^T||_F with C_i = Q_i R_i (no n x m product)."""
    T1 = np.linalg.qr(C1, mode="r")
    T2 = np.linalg.qr(C2, mode="r")
    return float(np.linalg.norm(T1 @ T2.T))

"""Final low-rank compression of a factored iterate X = V X^ W^T (test infrastructure only).

With orthonormal V, W (the FP64 block Arnoldi bases; deflated zero columns allowed, their
rows of X^ are zero) the singular values of X are those of X^ (Sec. 3.2: V, W column-
orthonormal), so X^ = U S Z^T gives X = (V U) S (W Z)^T.  Keeping the q largest singular
values, with q the smallest rank whose discarded part satisfies
sqrt(sum_{i > q} s_i^2) <= tol * ||S||_F, is the best rank-q approximation (Eckart-Young),
with ||X - X_q||_F equal to that discarded norm.
"""
from __future__ import annotations

import numpy as np


def truncation_rank(sv: np.ndarray, tol: float) -> int:
    """Smallest q with ||sv[q:]||_2 <= tol * ||sv||_2 (sv in descending order)."""
    total = np.sqrt(np.sum(sv**2))
    tail = np.sqrt(np.cumsum((sv**2)[::-1]))[::-1]  # tail[i] = ||sv[i:]||
    for q in range(len(sv) + 1):
        rest = tail[q] if q < len(sv) else 0.0
        if rest <= tol * total:
            return q
    return len(sv)


def compress(V: np.ndarray, Xh: np.ndarray, W: np.ndarray, tol: float):
    """Returns (V_q, s_q, W_q) with X ~ V_q diag(s_q) W_q^T."""
    U, sv, Zt = np.linalg.svd(Xh)
    q = truncation_rank(sv, tol)
    return V @ U[:, :q], sv[:q], W @ Zt[:q].T

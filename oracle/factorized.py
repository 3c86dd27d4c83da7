"""Factorized CG and BiCGSTAB (Algorithms 4.1, 4.2) and the Lyapunov variant (Sec. 4.3).

Test infrastructure only (see ``oracle/__init__``).  Plain numpy/scipy in
float64.  Iterates are kept as X = V X^ W^T with V, W orthonormal bases of the
block Krylov spaces K_k(A, C1) and K_k(B^T, C2) (Corollary 3.2) and X^ small.

Readings of points the paper leaves open (each also listed in the design notes):

* Thin QR of C1, C2 and of every new basis block: Householder (LAPACK via
  ``numpy.linalg.qr``) with the sign fixed so that diag(R) > 0, which makes
  the factors unique.
* Block Lanczos (Sec. 3.2, used by Algorithm 4.1): three-term recurrence in
  the order Y = A V_j - V_{j-1} H_{j-1,j}; H_{j,j} = V_j^T Y;
  Y -= V_j H_{j,j}; Y = V_{j+1} H_{j+1,j}, with H_{j-1,j} = H_{j,j-1}^T and
  no reorthogonalisation (the paper's per-step cost O(nnz s + n s^2) excludes
  it).
* Block Arnoldi (Sec. 3.2, used by Algorithm 4.2): block classical
  Gram-Schmidt applied twice (BCGS2): H1 = V^T Y, Y -= V H1, H2 = V^T Y,
  Y -= V H2, H_{:,j} = H1 + H2.
* Krylov exhaustion: with nu^2 = ||H_{1:j,j}||_F^2 + ||Y||_F^2 (Y after
  projection), a block with ||Y||_F <= delta * nu is replaced by a zero block
  and H_{j+1,j} = 0; all later blocks are zero too.  A partial rank loss
  (some diag(R) <= delta * nu but not all of Y) is a breakdown.
* The convergence test uses "<=" as the algorithms print it.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np


class Breakdown(Exception):
    pass


def thin_qr(Y: np.ndarray):
    """Y = Q R, Q with orthonormal columns, R upper triangular with diag(R) >= 0."""
    Q, R = np.linalg.qr(Y, mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :], R * d[:, None]


def deflating_qr(Y: np.ndarray, thr: float):
    """QR of a block whose columns may be (numerically) dependent: column by column, each
    column is orthogonalised twice against the columns kept so far; if what remains has norm
    <= thr the column is dropped (its Q column and its R row are zero, its R column keeps the
    coefficients on the kept columns, so Y = Q R still holds), otherwise it is normalised
    (diag(R) > 0).  The dropped columns stay zero in every later basis block (their images
    are zero), which keeps all shapes of Algorithms 4.1/4.2 and V X^ W^T unchanged."""
    n, s = Y.shape
    Q = np.zeros((n, s))
    R = np.zeros((s, s))
    kept = []
    for j in range(s):
        r = Y[:, j].copy()
        for _ in range(2):
            if kept:
                c = Q[:, kept].T @ r
                r -= Q[:, kept] @ c
                R[kept, j] += c
        nr = np.linalg.norm(r)
        if nr > thr:
            Q[:, j] = r / nr
            R[j, j] = nr
            kept.append(j)
    return Q, R


def pad(M: np.ndarray, t: int) -> np.ndarray:
    """[[M, O], [O, O]]: M in the top-left corner of a matrix t rows/cols larger."""
    out = np.zeros((M.shape[0] + t, M.shape[1] + t))
    out[: M.shape[0], : M.shape[1]] = M
    return out


def inner(X: np.ndarray, Y: np.ndarray) -> float:
    """<X, Y> = tr(X^T Y); equals the inner product of the large matrices (eq. 3.6)."""
    return float(np.sum(X * Y))


class BlockKrylovBasis:
    """Orthonormal basis V_k of K_k(A, C) with A V_k = V_{k+1} H_{k+1,k} (eq. 3.4).

    ``kind`` = "lanczos" (A symmetric, block tridiagonal H) or "arnoldi"
    (block upper Hessenberg H, BCGS2).  ``A`` is anything supporting ``A @ Y``.
    """

    def __init__(self, A, C: np.ndarray, kind: str, delta: float = 1e-12):
        self.A = A
        self.kind = kind
        self.delta = delta
        self.s = C.shape[1]
        V1, R = thin_qr(C)
        self.R0 = R  # C = V_1 R
        self.blocks: List[np.ndarray] = [V1]
        self.H = np.zeros((self.s, 0))  # H_{j+1, j} grows to (j+1)s x js
        self.exhausted = False
        self.deflated = 0  # basis columns dropped by partial losses of rank

    @property
    def nblocks(self) -> int:
        return len(self.blocks)

    def V(self, k: Optional[int] = None) -> np.ndarray:
        k = self.nblocks if k is None else k
        return np.hstack(self.blocks[:k])

    def Hk(self, rows: int, cols: int) -> np.ndarray:
        """H_{rows, cols} (block sizes), the leading (rows s) x (cols s) part."""
        return self.H[: rows * self.s, : cols * self.s]

    def step(self) -> None:
        """The j-th step: from V_j build V_{j+1} and the j-th block column of H."""
        s = self.s
        j = self.nblocks
        Hn = np.zeros(((j + 1) * s, j * s))
        Hn[: self.H.shape[0], : self.H.shape[1]] = self.H
        if self.exhausted:
            self.blocks.append(np.zeros_like(self.blocks[0]))
            self.H = Hn
            return
        Vj = self.blocks[j - 1]
        Y = np.asarray(self.A @ Vj, dtype=np.float64)
        if self.kind == "lanczos":
            if j >= 2:
                Hn[(j - 2) * s:(j - 1) * s, (j - 1) * s:j * s] = Hn[(j - 1) * s:j * s, (j - 2) * s:(j - 1) * s].T
                Y = Y - self.blocks[j - 2] @ Hn[(j - 2) * s:(j - 1) * s, (j - 1) * s:j * s]
            Hjj = Vj.T @ Y
            Y = Y - Vj @ Hjj
            Hn[(j - 1) * s:j * s, (j - 1) * s:j * s] = Hjj
        elif self.kind == "arnoldi":
            Vall = self.V(j)
            H1 = Vall.T @ Y
            Y = Y - Vall @ H1
            H2 = Vall.T @ Y
            Y = Y - Vall @ H2
            Hn[: j * s, (j - 1) * s:j * s] = H1 + H2
        else:
            raise ValueError(self.kind)
        ynorm = np.linalg.norm(Y)
        nu = np.sqrt(np.sum(Hn[: j * s, (j - 1) * s:j * s] ** 2) + ynorm**2)
        if ynorm <= self.delta * nu:
            self.exhausted = True
            self.blocks.append(np.zeros_like(Vj))
            self.H = Hn
            return
        Q, R = thin_qr(Y)
        if np.min(np.abs(np.diag(R))) <= self.delta * nu:
            # partial loss of rank: the dependent columns are deflated to zero columns
            Q, R = deflating_qr(Y, self.delta * nu)
            self.deflated += int(np.sum(np.diag(R) == 0.0))
        Hn[j * s:(j + 1) * s, (j - 1) * s:j * s] = R
        self.blocks.append(Q)
        self.H = Hn


def small_sylvester(H: np.ndarray, Z: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Factored Sylvester operator, eq. (3.7):

    A (V_k Z W_k^T) + (V_k Z W_k^T) B = V_{k+1} ([H Z, O] + [Z G^T; O]) W_{k+1}^T
    with H = H_{k+1,k}, G = G_{k+1,k} ((k+1)s x ks) and Z (ks x ks).
    """
    r = Z.shape[0]
    rp = H.shape[0]
    out = np.zeros((rp, rp))
    out[:, :r] += H @ Z
    out[:r, :] += Z @ G.T
    return out


def small_lyapunov(H: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """Sec. 4.3: with B = A^T, C2 = C1 and Z symmetric, [Z H^T; O] = [H Z, O]^T,
    so one product gives the operator: M + M^T with M = [H Z, O]."""
    r = Z.shape[0]
    rp = H.shape[0]
    M = np.zeros((rp, rp))
    M[:, :r] = H @ Z
    return M + M.T


@dataclasses.dataclass
class FactorizedResult:
    V: np.ndarray
    Xhat: np.ndarray
    W: np.ndarray
    iters: int
    status: str  # "converged" | "maxit" | "breakdown"
    history: List[float]
    Xhats: Optional[List[np.ndarray]] = None  # X^_k for k = 0.. (if kept)
    basisA: Optional[BlockKrylovBasis] = None
    basisB: Optional[BlockKrylovBasis] = None

    def X(self) -> np.ndarray:
        return self.V @ self.Xhat @ self.W.T

    def X_at(self, k: int, width_blocks: int) -> np.ndarray:
        """X_k = V X^_k W^T using the first ``width_blocks`` blocks of each basis."""
        V = self.basisA.V(width_blocks)
        W = (self.basisB or self.basisA).V(width_blocks)
        return V @ self.Xhats[k] @ W.T


def factorized_cg(A, B, C1: np.ndarray, C2: Optional[np.ndarray], tol: float, maxit: int,
                  lyapunov: bool = False, delta: float = 1e-12, keep_iterates: bool = False) -> FactorizedResult:
    """Algorithm 4.1 (A, B symmetric positive definite).

    With ``lyapunov`` (B = A^T, C2 = C1; pass B = None, C2 = None) one basis
    serves both sides and the operator is ``small_lyapunov`` (Sec. 4.3).
    Returns V_{k+1}, X^_{k+1}, W_{k+1} (width (k+1)s) at convergence.
    """
    s = C1.shape[1]
    bA = BlockKrylovBasis(A, C1, "lanczos", delta)
    bB = bA if lyapunov else BlockKrylovBasis(B.T, C2, "lanczos", delta)
    RL, RR = bA.R0, bB.R0
    Rh = RL @ RR.T
    if lyapunov:
        Rh = 0.5 * (Rh + Rh.T)
    Xh = np.zeros((0, 0))
    Ph = Rh.copy()
    rho = inner(Rh, Rh)
    r0 = np.sqrt(inner(Rh, Rh))
    hist = [1.0]
    xs = [Xh.copy()] if keep_iterates else None

    def result(k, status):
        w = Xh.shape[0] // s
        return FactorizedResult(bA.V(w), Xh, bB.V(w), k, status, hist, xs, bA, None if lyapunov else bB)

    for k in range(maxit):
        # block Lanczos step k+1 on both sides -> V_{k+2}, H_{k+2,k+1}
        try:
            bA.step()
            if not lyapunov:
                bB.step()
        except Breakdown:
            return result(k, "breakdown")
        H = bA.Hk(k + 2, k + 1)
        if lyapunov:
            Qh = small_lyapunov(H, Ph)
        else:
            Qh = small_sylvester(H, Ph, bB.Hk(k + 2, k + 1))
        r = (k + 1) * s
        pq = inner(Ph, Qh[:r, :r])
        if not np.isfinite(pq) or pq <= 0.0:
            return result(k, "breakdown")
        alpha = rho / pq
        Xh = pad(Xh, s) + alpha * Ph
        Rh = pad(Rh, s) - alpha * Qh
        rn = np.sqrt(inner(Rh, Rh))
        hist.append(rn / r0)
        if xs is not None:
            xs.append(Xh.copy())
        if not np.isfinite(rn):
            return result(k + 1, "breakdown")
        if rn <= r0 * tol:
            return result(k + 1, "converged")
        rho_new = inner(Rh, Rh)
        beta = rho_new / rho
        rho = rho_new
        Ph = Rh + pad(beta * Ph, s)
    return result(maxit, "maxit")


def factorized_bicgstab(A, B, C1: np.ndarray, C2: np.ndarray, tol: float, maxit: int, delta: float = 1e-12,
                        keep_iterates: bool = False, callback=None) -> FactorizedResult:
    """Algorithm 4.2 (general A, B; block Arnoldi bases).

    Returns V_{2k+2}, X^_{k+1}, W_{2k+2} (width (2k+2)s) at convergence.
    """
    s = C1.shape[1]
    bA = BlockKrylovBasis(A, C1, "arnoldi", delta)
    bB = BlockKrylovBasis(B.T, C2, "arnoldi", delta)
    Rh = bA.R0 @ bB.R0.T
    Ph = Rh.copy()
    Rt = Rh.copy()  # shadow residual R~_0 (s x s)
    rho = inner(Rt, Rh)
    Xh = np.zeros((0, 0))
    r0 = np.sqrt(inner(Rh, Rh))
    hist = [1.0]
    xs = [Xh.copy()] if keep_iterates else None

    def result(k, status):
        w = Xh.shape[0] // s
        return FactorizedResult(bA.V(w), Xh, bB.V(w), k, status, hist, xs, bA, bB)

    for k in range(maxit):
        # Arnoldi step 2k+1 on both sides -> V_{2k+2}, H_{2k+2,2k+1}
        try:
            bA.step()
            bB.step()
        except Breakdown:
            return result(k, "breakdown")
        Qh = small_sylvester(bA.Hk(2 * k + 2, 2 * k + 1), Ph, bB.Hk(2 * k + 2, 2 * k + 1))
        d = inner(Rt, Qh[:s, :s])
        if not np.isfinite(d) or d == 0.0:
            return result(k, "breakdown")
        alpha = rho / d
        Sh = pad(Rh, s) - alpha * Qh
        # Arnoldi step 2k+2 -> V_{2k+3}, H_{2k+3,2k+2}
        try:
            bA.step()
            bB.step()
        except Breakdown:
            return result(k, "breakdown")
        Th = small_sylvester(bA.Hk(2 * k + 3, 2 * k + 2), Sh, bB.Hk(2 * k + 3, 2 * k + 2))
        rs = (2 * k + 2) * s
        tt = inner(Th, Th)
        if not np.isfinite(tt) or tt == 0.0:
            return result(k, "breakdown")
        omega = inner(Th[:rs, :rs], Sh) / tt
        if omega == 0.0:
            return result(k, "breakdown")
        Xh = pad(Xh, 2 * s) + pad(alpha * Ph, s) + omega * Sh
        Rh = pad(Sh, s) - omega * Th
        rn = np.sqrt(inner(Rh, Rh))
        hist.append(rn / r0)
        if callback is not None:
            callback(k + 1, rn / r0)
        if xs is not None:
            xs.append(Xh.copy())
        if not np.isfinite(rn):
            return result(k + 1, "breakdown")
        if rn <= r0 * tol:
            return result(k + 1, "converged")
        rho_new = inner(Rt, Rh[:s, :s])
        if rho_new == 0.0:
            return result(k + 1, "breakdown")
        beta = (alpha / omega) * (rho_new / rho)
        rho = rho_new
        Ph = Rh + beta * (pad(Ph, 2 * s) - omega * pad(Qh, s))
    return result(maxit, "maxit")


def factorized_cgs(A, B, C1: np.ndarray, C2: np.ndarray, tol: float, maxit: int, delta: float = 1e-12,
                   keep_iterates: bool = False) -> FactorizedResult:
    """Factorized CGS: ``matrix_oriented.cgs`` with every iterate kept as V X^ W^T on block
    Arnoldi bases, built the way Sec. 4.2 builds Algorithm 4.2 from Algorithm 2.2 (Sec. 4
    states the approach carries over to CGS; the paper prints no listing for it).

    With the iterates R_k, U_k, P_k on the first 2k+1 blocks, each iteration takes two
    Arnoldi steps per side: L(P_k) needs V_{2k+2} (eq. 3.7), Q_k and U_k + Q_k live there,
    and L(U_k + Q_k) needs V_{2k+3}.  Additions are additions of the zero-padded small
    matrices (eq. 3.5); R~_0 = R_0 lives in the first block, so <R~_0, M> is the inner
    product with the leading s x s block of M^ (eq. 3.6).  Returns V_{2k+2}, X^_{k+1},
    W_{2k+2} (width (2k+2)s), the shapes of Algorithm 4.2.
    """
    s = C1.shape[1]
    bA = BlockKrylovBasis(A, C1, "arnoldi", delta)
    bB = BlockKrylovBasis(B.T, C2, "arnoldi", delta)
    Rh = bA.R0 @ bB.R0.T
    Rt = Rh.copy()  # shadow residual R~_0 (s x s)
    Uh = Rh.copy()
    Ph = Rh.copy()
    rho = inner(Rt, Rh)
    Xh = np.zeros((0, 0))
    r0 = np.sqrt(inner(Rh, Rh))
    hist = [1.0]
    xs = [Xh.copy()] if keep_iterates else None

    def result(k, status):
        w = Xh.shape[0] // s
        return FactorizedResult(bA.V(w), Xh, bB.V(w), k, status, hist, xs, bA, bB)

    for k in range(maxit):
        # Arnoldi step 2k+1 on both sides -> V_{2k+2}: L(P_k)
        try:
            bA.step()
            bB.step()
        except Breakdown:
            return result(k, "breakdown")
        Vh = small_sylvester(bA.Hk(2 * k + 2, 2 * k + 1), Ph, bB.Hk(2 * k + 2, 2 * k + 1))
        d = inner(Rt, Vh[:s, :s])
        if not np.isfinite(d) or d == 0.0:
            return result(k, "breakdown")
        alpha = rho / d
        Qh = pad(Uh, s) - alpha * Vh
        Wh = pad(Uh, s) + Qh
        Xh = pad(Xh, 2 * s) + alpha * Wh
        # Arnoldi step 2k+2 -> V_{2k+3}: L(U_k + Q_k)
        try:
            bA.step()
            bB.step()
        except Breakdown:
            return result(k, "breakdown")
        Th = small_sylvester(bA.Hk(2 * k + 3, 2 * k + 2), Wh, bB.Hk(2 * k + 3, 2 * k + 2))
        Rh = pad(Rh, 2 * s) - alpha * Th
        rn = np.sqrt(inner(Rh, Rh))
        hist.append(rn / r0)
        if xs is not None:
            xs.append(Xh.copy())
        if not np.isfinite(rn):
            return result(k + 1, "breakdown")
        if rn <= r0 * tol:
            return result(k + 1, "converged")
        rho_new = inner(Rt, Rh[:s, :s])
        if rho_new == 0.0:
            return result(k + 1, "breakdown")
        beta = rho_new / rho
        rho = rho_new
        Uh = Rh + beta * pad(Qh, s)
        Ph = Uh + beta * (pad(Qh, s) + beta * pad(Ph, 2 * s))
    return result(maxit, "maxit")


def factorized_cr(A, B, C1: np.ndarray, C2: Optional[np.ndarray], tol: float, maxit: int,
                  lyapunov: bool = False, delta: float = 1e-12, keep_iterates: bool = False) -> FactorizedResult:
    """Factorized CR: ``matrix_oriented.cr`` with every iterate kept as V X^ W^T on block
    Lanczos bases (A, B symmetric), built the way Sec. 4.1 builds Algorithm 4.1 from
    Algorithm 2.1 (Sec. 4 states the approach carries over to CR; the paper prints no listing).

    R_k lives on the first k+1 blocks and L(R_k), L(P_k) on k+2 (eq. 3.7), so each iteration
    takes one Lanczos step per side, after the convergence test, for L(R_{k+1}); one more
    step before the loop gives L(R_0).  Inner products of padded small matrices (eq. 3.6);
    with ``lyapunov`` one basis and the operator of Sec. 4.3.  Returns V_{k+1}, X^_{k+1},
    W_{k+1} (width (k+1)s), the shapes of Algorithm 4.1.
    """
    s = C1.shape[1]
    bA = BlockKrylovBasis(A, C1, "lanczos", delta)
    bB = bA if lyapunov else BlockKrylovBasis(B.T, C2, "lanczos", delta)
    Rh = bA.R0 @ bB.R0.T
    if lyapunov:
        Rh = 0.5 * (Rh + Rh.T)
    Xh = np.zeros((0, 0))
    r0 = np.sqrt(inner(Rh, Rh))
    hist = [1.0]
    xs = [Xh.copy()] if keep_iterates else None

    def result(k, status):
        w = Xh.shape[0] // s
        return FactorizedResult(bA.V(w), Xh, bB.V(w), k, status, hist, xs, bA, None if lyapunov else bB)

    def op(j, Z):  # L(V_j Z W_j^T) on blocks 1..j+1 (eq. 3.7)
        H = bA.Hk(j + 1, j)
        return small_lyapunov(H, Z) if lyapunov else small_sylvester(H, Z, bB.Hk(j + 1, j))

    def step():
        bA.step()
        if not lyapunov:
            bB.step()

    try:
        step()  # V_2: L(R_0)
    except Breakdown:
        return result(0, "breakdown")
    LRh = op(1, Rh)
    rho = inner(Rh, LRh[:s, :s])
    Ph, LPh = Rh.copy(), LRh.copy()
    for k in range(maxit):
        lp = inner(LPh, LPh)
        if not np.isfinite(rho) or rho == 0.0 or not np.isfinite(lp) or lp == 0.0:
            return result(k, "breakdown")
        alpha = rho / lp
        Xh = pad(Xh, s) + alpha * Ph
        Rh = pad(Rh, s) - alpha * LPh
        rn = np.sqrt(inner(Rh, Rh))
        hist.append(rn / r0)
        if xs is not None:
            xs.append(Xh.copy())
        if not np.isfinite(rn):
            return result(k + 1, "breakdown")
        if rn <= r0 * tol:
            return result(k + 1, "converged")
        try:
            step()  # V_{k+3}: L(R_{k+1})
        except Breakdown:
            return result(k + 1, "breakdown")
        LRh = op(k + 2, Rh)
        r = (k + 2) * s
        rho_new = inner(Rh, LRh[:r, :r])
        beta = rho_new / rho
        rho = rho_new
        Ph = Rh + beta * pad(Ph, s)
        LPh = LRh + beta * pad(LPh, s)
    return result(maxit, "maxit")


def pad_to(M: np.ndarray, e: int) -> np.ndarray:
    """M in the top-left corner of an e x e zero matrix (M is at most e x e)."""
    return pad(M, e - M.shape[0]) if M.shape[0] <= e else M


def factorized_gpbicg(A, B, C1: np.ndarray, C2: np.ndarray, tol: float, maxit: int, delta: float = 1e-12,
                      keep_iterates: bool = False) -> FactorizedResult:
    """Factorized GPBiCG: ``matrix_oriented.gpbicg`` with every iterate kept as V M^ W^T on
    block Arnoldi bases, built the way Sec. 4.2 builds Algorithm 4.2 (Sec. 4 states the
    approach carries over to GPBiCG; the paper prints no listing).

    With R_n on the first 2n+1 blocks, L(P_n) (eq. 3.7) needs V_{2n+2} and L(T_n) needs
    V_{2n+3}: two Arnoldi steps per iteration, as BiCGSTAB.  Extents: P, R on (2n+1)s; L(P),
    T, Y, U, Z and X on (2n+2)s; L(T), W and the new R on (2n+3)s.  Additions of zero-padded
    small matrices (eq. 3.5), inner products of small matrices (eq. 3.6; <R~_0, M> on the
    leading s x s block).  Returns V_{2k+2}, X^_{k+1}, W_{2k+2} like Algorithm 4.2.
    """
    s = C1.shape[1]
    bA = BlockKrylovBasis(A, C1, "arnoldi", delta)
    bB = BlockKrylovBasis(B.T, C2, "arnoldi", delta)
    Rh = bA.R0 @ bB.R0.T
    Rt = Rh.copy()
    z = np.zeros((0, 0))
    Ph, Uh, Wh, Zh, Tph, Xh = z, z, z, z, z, z
    beta = 0.0
    rho = inner(Rt, Rh)
    r0 = np.sqrt(inner(Rh, Rh))
    hist = [1.0]
    xs = [Xh.copy()] if keep_iterates else None

    def result(k, status):
        w = Xh.shape[0] // s
        return FactorizedResult(bA.V(w), Xh, bB.V(w), k, status, hist, xs, bA, bB)

    for k in range(maxit):
        e1, e2, e3 = (2 * k + 1) * s, (2 * k + 2) * s, (2 * k + 3) * s
        Ph = pad_to(Rh, e1) + beta * (pad_to(Ph, e1) - pad_to(Uh, e1))
        try:  # Arnoldi step 2k+1 -> V_{2k+2}: L(P)
            bA.step()
            bB.step()
        except Breakdown:
            return result(k, "breakdown")
        LPh = small_sylvester(bA.Hk(2 * k + 2, 2 * k + 1), Ph, bB.Hk(2 * k + 2, 2 * k + 1))
        d = inner(Rt, LPh[:s, :s])
        if not np.isfinite(d) or d == 0.0:
            return result(k, "breakdown")
        alpha = rho / d
        Yh = pad_to(Tph, e2) - pad_to(Rh, e2) - alpha * pad_to(Wh, e2) + alpha * LPh
        Th = pad_to(Rh, e2) - alpha * LPh
        try:  # Arnoldi step 2k+2 -> V_{2k+3}: L(T)
            bA.step()
            bB.step()
        except Breakdown:
            return result(k, "breakdown")
        LTh = small_sylvester(bA.Hk(2 * k + 3, 2 * k + 2), Th, bB.Hk(2 * k + 3, 2 * k + 2))
        if k == 0:
            aa = inner(LTh, LTh)
            if not np.isfinite(aa) or aa == 0.0:
                return result(k, "breakdown")
            zeta, eta = inner(LTh[:e2, :e2], Th) / aa, 0.0
        else:
            yy, tt_, yt = inner(Yh, Yh), inner(LTh[:e2, :e2], Th), inner(Yh, Th)
            ty, aa = inner(LTh[:e2, :e2], Yh), inner(LTh, LTh)
            den = aa * yy - ty * ty
            if not np.isfinite(den) or den == 0.0:
                return result(k, "breakdown")
            zeta = (yy * tt_ - yt * ty) / den
            eta = (aa * yt - ty * tt_) / den
        if zeta == 0.0:
            return result(k, "breakdown")
        Uh = zeta * LPh + eta * (pad_to(Tph, e2) - pad_to(Rh, e2) + beta * pad_to(Uh, e2))
        Zh = zeta * pad_to(Rh, e2) + eta * pad_to(Zh, e2) - alpha * Uh
        Xh = pad_to(Xh, e2) + alpha * pad_to(Ph, e2) + Zh
        Rh = pad_to(Th, e3) - eta * pad_to(Yh, e3) - zeta * LTh
        rn = np.sqrt(inner(Rh, Rh))
        hist.append(rn / r0)
        if xs is not None:
            xs.append(Xh.copy())
        if not np.isfinite(rn):
            return result(k + 1, "breakdown")
        if rn <= r0 * tol:
            return result(k + 1, "converged")
        rho_new = inner(Rt, Rh[:s, :s])
        if rho_new == 0.0:
            return result(k + 1, "breakdown")
        beta = (alpha / zeta) * (rho_new / rho)
        rho = rho_new
        Wh = LTh + beta * pad_to(LPh, e3)
        Tph = Th
    return result(maxit, "maxit")

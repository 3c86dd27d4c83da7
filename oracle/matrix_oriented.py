"""Matrix-oriented CG, BiCGSTAB, CGS, CR and GPBiCG on full n x m iterates (Algorithms 2.1,
2.2; CGS, CR and GPBiCG as Sec. 4 names them: Sonneveld 1989, Stiefel 1955, Zhang 1997).

Test infrastructure only (see ``oracle/__init__``).  These are the plain
definitions that the factorized methods are mathematically equivalent to
(Sec. 5.1): every vector operation of CG / BiCGSTAB on the Kronecker system
(eq. 1.2) is done on the n x m matrix it represents (Sec. 2):
addition -> matrix addition, inner product -> <X, Y> = tr(X^T Y),
matrix-vector product -> the Sylvester operator A X + X B.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np


def sylvester_op(A, B, X: np.ndarray) -> np.ndarray:
    """A X + X B (the Sylvester operator, Sec. 2).  A, B scipy sparse or dense."""
    return np.asarray(A @ X) + np.asarray((B.T @ X.T).T)


def inner(X: np.ndarray, Y: np.ndarray) -> float:
    """<X, Y> = tr(X^T Y) (Sec. 2)."""
    return float(np.sum(X * Y))


@dataclasses.dataclass
class FullResult:
    X: np.ndarray
    iters: int
    status: str
    history: List[float]
    iterates: Optional[List[np.ndarray]] = None


def cg(A, B, C: np.ndarray, tol: float, maxit: int, keep_iterates: bool = False) -> FullResult:
    """Algorithm 2.1 with X_0 = 0 (Sec. 4.1).

    Stops at the first k with ||R_{k+1}|| <= ||R_0|| tol and returns X_{k+1};
    otherwise returns X_maxit with status "maxit".
    """
    X = np.zeros_like(C)
    R = C - sylvester_op(A, B, X)
    P = R.copy()
    rho = inner(R, R)
    r0 = np.linalg.norm(R)
    hist = [1.0]
    its = [X.copy()] if keep_iterates else None
    for k in range(maxit):
        Q = sylvester_op(A, B, P)            # Q_k = A P_k + P_k B
        alpha = rho / inner(P, Q)
        X = X + alpha * P
        R = R - alpha * Q
        rn = np.linalg.norm(R)
        hist.append(rn / r0)
        if its is not None:
            its.append(X.copy())
        if rn <= r0 * tol:
            return FullResult(X, k + 1, "converged", hist, its)
        rho_new = inner(R, R)
        beta = rho_new / rho
        rho = rho_new
        P = R + beta * P
    return FullResult(X, maxit, "maxit", hist, its)


def bicgstab(A, B, C: np.ndarray, tol: float, maxit: int, keep_iterates: bool = False) -> FullResult:
    """Algorithm 2.2 with X_0 = 0 and the shadow residual R~_0 = R_0."""
    X = np.zeros_like(C)
    R = C - sylvester_op(A, B, X)
    Rt = R.copy()
    P = R.copy()
    rho = inner(R, Rt)
    r0 = np.linalg.norm(R)
    hist = [1.0]
    its = [X.copy()] if keep_iterates else None
    for k in range(maxit):
        Q = sylvester_op(A, B, P)            # Q_k = A P_k + P_k B
        alpha = rho / inner(Rt, Q)
        S = R - alpha * Q
        T = sylvester_op(A, B, S)            # T_k = A S_k + S_k B
        omega = inner(T, S) / inner(T, T)
        X = X + alpha * P + omega * S
        R = S - omega * T
        rn = np.linalg.norm(R)
        hist.append(rn / r0)
        if its is not None:
            its.append(X.copy())
        if rn <= r0 * tol:
            return FullResult(X, k + 1, "converged", hist, its)
        rho_new = inner(R, Rt)
        beta = alpha / omega * rho_new / rho
        rho = rho_new
        P = R + beta * (P - omega * Q)
    return FullResult(X, maxit, "maxit", hist, its)


def cgs(A, B, C: np.ndarray, tol: float, maxit: int, keep_iterates: bool = False) -> FullResult:
    """Conjugate Gradient Squared (Sonneveld 1989) on the Kronecker system (eq. 1.2), written
    with the matrix operations of Sec. 2, X_0 = 0, shadow residual R~_0 = R_0.  Sec. 4 names
    CGS among the methods the factorized approach applies to; the paper gives no algorithm
    listing for it, so this is the textbook recurrence with its vectors read as n x m matrices:

        alpha = rho_k / <R~_0, L(P_k)>,  Q_k = U_k - alpha L(P_k),
        X_{k+1} = X_k + alpha (U_k + Q_k),  R_{k+1} = R_k - alpha L(U_k + Q_k),
        beta = rho_{k+1} / rho_k,  U_{k+1} = R_{k+1} + beta Q_k,
        P_{k+1} = U_{k+1} + beta (Q_k + beta P_k),    L(Y) = A Y + Y B.
    """
    X = np.zeros_like(C)
    R = C - sylvester_op(A, B, X)
    Rt = R.copy()
    U = R.copy()
    P = R.copy()
    rho = inner(Rt, R)
    r0 = np.linalg.norm(R)
    hist = [1.0]
    its = [X.copy()] if keep_iterates else None
    for k in range(maxit):
        V = sylvester_op(A, B, P)
        alpha = rho / inner(Rt, V)
        Q = U - alpha * V
        W = U + Q
        X = X + alpha * W
        R = R - alpha * sylvester_op(A, B, W)
        rn = np.linalg.norm(R)
        hist.append(rn / r0)
        if its is not None:
            its.append(X.copy())
        if rn <= r0 * tol:
            return FullResult(X, k + 1, "converged", hist, its)
        rho_new = inner(Rt, R)
        beta = rho_new / rho
        rho = rho_new
        U = R + beta * Q
        P = U + beta * (Q + beta * P)
    return FullResult(X, maxit, "maxit", hist, its)


def cr(A, B, C: np.ndarray, tol: float, maxit: int, keep_iterates: bool = False) -> FullResult:
    """Conjugate Residual (Stiefel 1955) on the Kronecker system (eq. 1.2) with A, B symmetric,
    so that L(Y) = A Y + Y B is self-adjoint for <., .> (Sec. 2); X_0 = 0.  Sec. 4 names CR
    among the methods the factorized approach applies to; the paper gives no listing, so this
    is the textbook recurrence with its vectors read as n x m matrices:

        alpha = <R_k, L(R_k)> / <L(P_k), L(P_k)>,  X_{k+1} = X_k + alpha P_k,
        R_{k+1} = R_k - alpha L(P_k),  beta = <R_{k+1}, L(R_{k+1})> / <R_k, L(R_k)>,
        P_{k+1} = R_{k+1} + beta P_k,  L(P_{k+1}) = L(R_{k+1}) + beta L(P_k).
    """
    X = np.zeros_like(C)
    R = C - sylvester_op(A, B, X)
    LR = sylvester_op(A, B, R)
    P, LP = R.copy(), LR.copy()
    rho = inner(R, LR)
    r0 = np.linalg.norm(R)
    hist = [1.0]
    its = [X.copy()] if keep_iterates else None
    for k in range(maxit):
        alpha = rho / inner(LP, LP)
        X = X + alpha * P
        R = R - alpha * LP
        rn = np.linalg.norm(R)
        hist.append(rn / r0)
        if its is not None:
            its.append(X.copy())
        if rn <= r0 * tol:
            return FullResult(X, k + 1, "converged", hist, its)
        LR = sylvester_op(A, B, R)
        rho_new = inner(R, LR)
        beta = rho_new / rho
        rho = rho_new
        P = R + beta * P
        LP = LR + beta * LP
    return FullResult(X, maxit, "maxit", hist, its)


def gpbicg(A, B, C: np.ndarray, tol: float, maxit: int, keep_iterates: bool = False,
           eta_zero: bool = False, record: Optional[list] = None) -> FullResult:
    """GPBiCG (Zhang 1997, generalized product-type BiCG) on the Kronecker system (eq. 1.2) in
    the matrix operations of Sec. 2, X_0 = 0, R~_0 = R_0.  Sec. 4 names GPBiCG among the
    methods the factorized approach applies to; the paper gives no listing, so this is the
    published recurrence with its vectors read as n x m matrices.  Per iteration, with
    L(Y) = A Y + Y B:

        P = R + beta (P - U),  alpha = <R~_0, R> / <R~_0, L(P)>,
        Y = T_prev - R - alpha W + alpha L(P),  T = R - alpha L(P),
        (zeta, eta) minimise ||T - zeta L(T) - eta Y||  (eta = 0 in the first iteration),
        U = zeta L(P) + eta (T_prev - R + beta U),  Z = zeta R + eta Z - alpha U,
        X = X + alpha P + Z,  R = T - eta Y - zeta L(T),
        beta = (alpha / zeta) <R~_0, R_new> / <R~_0, R_old>,  W = L(T) + beta L(P),  T_prev = T.

    With ``eta_zero`` every eta is 0 and the recurrence is BiCGSTAB's (omega = zeta): a pin.
    ``record`` (a list) receives (R_new, L(T), Y) of every iteration.
    """
    X = np.zeros_like(C)
    R = C - sylvester_op(A, B, X)
    Rt = R.copy()
    P = np.zeros_like(C)
    U = np.zeros_like(C)
    W = np.zeros_like(C)
    Z = np.zeros_like(C)
    Tp = np.zeros_like(C)
    beta = 0.0
    rho = inner(Rt, R)
    r0 = np.linalg.norm(R)
    hist = [1.0]
    its = [X.copy()] if keep_iterates else None
    for k in range(maxit):
        P = R + beta * (P - U)
        LP = sylvester_op(A, B, P)
        alpha = rho / inner(Rt, LP)
        Y = Tp - R - alpha * W + alpha * LP
        T = R - alpha * LP
        LT = sylvester_op(A, B, T)
        if k == 0 or eta_zero:
            zeta = inner(LT, T) / inner(LT, LT)
            eta = 0.0
        else:
            yy, tt_, yt = inner(Y, Y), inner(LT, T), inner(Y, T)
            ty, aa = inner(LT, Y), inner(LT, LT)
            den = aa * yy - ty * ty
            zeta = (yy * tt_ - yt * ty) / den
            eta = (aa * yt - ty * tt_) / den
        U = zeta * LP + eta * (Tp - R + beta * U)
        Z = zeta * R + eta * Z - alpha * U
        X = X + alpha * P + Z
        R = T - eta * Y - zeta * LT
        if record is not None:
            record.append((R.copy(), LT, Y))
        rn = np.linalg.norm(R)
        hist.append(rn / r0)
        if its is not None:
            its.append(X.copy())
        if rn <= r0 * tol:
            return FullResult(X, k + 1, "converged", hist, its)
        rho_new = inner(Rt, R)
        beta = (alpha / zeta) * (rho_new / rho)
        rho = rho_new
        W = LT + beta * LP
        Tp = T
    return FullResult(X, maxit, "maxit", hist, its)

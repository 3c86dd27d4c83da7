"""Seeded synthetic inputs for the Sylvester equation A X + X B = C1 C2^T.

This module only builds inputs: sparse operators in CSR form and random
right-hand-side factors.  It holds none of the solver arithmetic, so both the
CPU oracle (``oracle/``) and the CUDA path (through its tests and ``bench.py``)
draw their inputs from here.

The paper's test matrices come from an earlier study that is not reproduced in
the paper (Sec. 5, Examples 5.1-5.4: a 2D finite-difference Laplacian for the
Lyapunov/CG experiments and a 3D convection-diffusion operator for the
Sylvester/BiCGSTAB experiments; C "chosen randomly").  The generators below are
stand-ins with the same structure:

* ``laplacian_2d(N)``: 5-point stencil on an N x N grid, lexicographic index
  ``i + N*j``, diagonal 4, neighbours -1 (no h^-2 factor).  Symmetric positive
  definite; eigenvalues 4 - 2cos(p*pi/(N+1)) - 2cos(q*pi/(N+1)).
* ``convdiff_3d(N, seed)``: -nu*Lap(u) + w.grad(u) on (0,1)^3 with zero
  Dirichlet boundary, h = 1/(N+1), nu = 1, |w| = 10 (global Peclet number
  |w| L / nu = 10), direction d = g/|g| with g ~ N(0, I_3) drawn from
  ``numpy.random.default_rng(seed)``; first-order upwind convection; the matrix
  is h^2 times the discrete operator.  Diagonal 6 + h*sum|w_c|, -e_c neighbour
  -1 - h*max(w_c, 0), +e_c neighbour -1 + h*min(w_c, 0): an irreducibly
  diagonally dominant M-matrix.
* ``rhs(n, m, s, seed)``: C1 (n x s) then C2 (m x s), i.i.d. N(0,1) from
  ``default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class CSR:
    """0-based CSR matrix with int32 indices and float64 values."""

    nrows: int
    ncols: int
    row_ptr: np.ndarray  # int32, nrows + 1
    col_idx: np.ndarray  # int32, nnz
    val: np.ndarray  # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.nrows, self.ncols))

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.nrows, self.ncols))
        for i in range(self.nrows):
            for p in range(self.row_ptr[i], self.row_ptr[i + 1]):
                out[i, self.col_idx[p]] += self.val[p]
        return out

    def transpose(self) -> "CSR":
        """Explicit transpose (used to build B^T from B)."""
        rows = np.repeat(np.arange(self.nrows, dtype=np.int64), np.diff(self.row_ptr))
        order = np.lexsort((rows, self.col_idx))
        cnt = np.bincount(self.col_idx, minlength=self.ncols)
        rp = np.zeros(self.ncols + 1, dtype=np.int64)
        rp[1:] = np.cumsum(cnt)
        return CSR(self.ncols, self.nrows, rp.astype(np.int32), rows[order].astype(np.int32),
                   self.val[order].copy())


def _from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    cnt = np.bincount(rows, minlength=n)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(cnt)
    return CSR(n, n, rp.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64))


def stencil_csr(shape, diag, offsets_vals) -> CSR:
    """CSR of a constant-coefficient stencil on a tensor grid, zero Dirichlet.

    ``shape`` = (N0, N1, ...) with axis 0 fastest (lexicographic index
    i0 + N0*(i1 + N1*i2 ...)); ``offsets_vals`` is a list of ((axis, step),
    value) pairs.
    """
    shape = tuple(int(x) for x in shape)
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for N in shape:
        coords.append(rem % N)
        rem //= N
    strides = [1]
    for N in shape[:-1]:
        strides.append(strides[-1] * N)
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, float(diag))]
    for (axis, step), v in offsets_vals:
        c = coords[axis] + step
        ok = (c >= 0) & (c < shape[axis])
        rows.append(idx[ok])
        cols.append(idx[ok] + step * strides[axis])
        vals.append(np.full(int(ok.sum()), float(v)))
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def laplacian_2d(N: int, shift: float = 0.0) -> CSR:
    """5-point Laplacian on an N x N grid (diag 4 + shift, neighbours -1)."""
    offs = [((0, -1), -1.0), ((0, 1), -1.0), ((1, -1), -1.0), ((1, 1), -1.0)]
    return stencil_csr((N, N), 4.0 + shift, offs)


def wind_direction(seed: int) -> np.ndarray:
    g = np.random.default_rng(seed).standard_normal(3)
    return g / np.linalg.norm(g)


def convdiff_3d(N: int, seed: int, peclet: float = 10.0, nu: float = 1.0) -> CSR:
    """h^2-scaled first-order upwind -nu Lap(u) + w.grad(u) on an N^3 grid."""
    h = 1.0 / (N + 1)
    w = peclet * nu * wind_direction(seed)  # |w| L / nu = peclet with L = 1
    diag = 6.0 * nu + h * float(np.abs(w).sum())
    offs = []
    for c in range(3):
        offs.append(((c, -1), -nu - h * max(w[c], 0.0)))
        offs.append(((c, 1), -nu + h * min(w[c], 0.0)))
    return stencil_csr((N, N, N), diag, offs)


def diagonal(d: np.ndarray) -> CSR:
    n = d.shape[0]
    return CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
               np.asarray(d, dtype=np.float64).copy())


def random_sparse(n: int, nnz_per_row: int, seed: int, spd: bool = False, diag_boost: float = 0.0) -> CSR:
    """Random sparse matrix with a ragged row-length mix (for kernel edge cases).

    Row i has between 0 and 2*nnz_per_row off-diagonal entries plus a
    diagonal.  With ``spd`` the matrix is symmetrised and made strictly
    diagonally dominant.
    """
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, 2 * nnz_per_row + 1, size=n)
    rows = np.repeat(np.arange(n), lens)
    cols = rng.integers(0, n, size=rows.shape[0])
    vals = rng.standard_normal(rows.shape[0])
    if spd:
        rows, cols = np.concatenate([rows, cols]), np.concatenate([cols, rows])
        vals = np.concatenate([vals, vals])
    keep = rows != cols
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    # merge duplicates
    key = rows.astype(np.int64) * n + cols
    uk, inv = np.unique(key, return_inverse=True)
    v = np.zeros(uk.shape[0])
    np.add.at(v, inv, vals)
    rows, cols = (uk // n).astype(np.int64), (uk % n).astype(np.int64)
    absrow = np.zeros(n)
    np.add.at(absrow, rows, np.abs(v))
    d = absrow + 1.0 + diag_boost
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    v = np.concatenate([v, d])
    return _from_coo(n, rows, cols, v)


def rhs(n: int, m: Optional[int], s: int, seed: int = 0):
    """C1 (n x s) then C2 (m x s), i.i.d. N(0,1), C order fill.  m=None: C2 = C1."""
    rng = np.random.default_rng(seed)
    C1 = rng.standard_normal((n, s))
    C2 = C1.copy() if m is None else rng.standard_normal((m, s))
    return C1, C2


@dataclasses.dataclass
class Problem:
    name: str
    A: CSR
    B: Optional[CSR]  # None in the Lyapunov case (B = A^T)
    C1: np.ndarray
    C2: Optional[np.ndarray]  # None in the Lyapunov case (C2 = C1)
    s: int
    method: str  # "cg" | "bicgstab"
    tol: float
    maxit: int
    precision: str = "fp64"  # "fp64" | "mixed"
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def lyapunov(self) -> bool:
        return self.B is None

    def B_eff(self) -> CSR:
        return self.A.transpose() if self.B is None else self.B

    def C2_eff(self) -> np.ndarray:
        return self.C1 if self.C2 is None else self.C2


def cfg_laplace_cg(N: int = 20, s: int = 1, seed: int = 0, tol: float = 1e-8, maxit: int = 200,
                   precision: str = "fp64") -> Problem:
    """Factorized CG, A = B = 5-point Laplacian (n = m = N^2), C1, C2 ~ N(0,1) seed 0.

    N = 20, s = 1 is the 400-unknown parity workload; s = 8 in mixed precision
    is the Krylov-exhaustion workload.
    """
    A = laplacian_2d(N)
    B = laplacian_2d(N)
    C1, C2 = rhs(A.nrows, B.nrows, s, seed)
    return Problem(f"laplace2d_N{N}_s{s}_cg_{precision}", A, B, C1, C2, s, "cg", tol, maxit, precision,
                   {"N": N})


def cfg_convdiff_bicgstab(NA: int = 64, NB: int = 48, s: int = 4, seed: int = 0, tol: float = 1e-8,
                          maxit: int = 300, precision: str = "fp64") -> Problem:
    """Factorized BiCGSTAB, A = CD NA^3 (wind seed 1), B = CD NB^3 (wind seed 2)."""
    A = convdiff_3d(NA, 1)
    B = convdiff_3d(NB, 2)
    C1, C2 = rhs(A.nrows, B.nrows, s, seed)
    return Problem(f"convdiff3d_{NA}x{NB}_s{s}_bicgstab_{precision}", A, B, C1, C2, s, "bicgstab", tol, maxit,
                   precision, {"NA": NA, "NB": NB, "windA": wind_direction(1).tolist(),
                               "windB": wind_direction(2).tolist()})


def cfg_batched_lyapunov(count: int = 64, seed: int = 4, Nmin: int = 64, Nmax: int = 256, tol: float = 1e-8,
                         maxit: int = 1000, s_choices=(1, 2, 4)) -> List[Problem]:
    """Batched Lyapunov CG instances: A = L_N + sigma*I, N ~ U{Nmin..Nmax}, s ~ {1,2,4}, sigma ~ U[0,1].

    One ``default_rng(seed)`` stream draws, per instance in order: N, s,
    sigma, then C1 (N^2 x s).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.integers(Nmin, Nmax + 1))
        s = int(rng.choice(np.asarray(s_choices)))
        sigma = float(rng.random())
        C1 = rng.standard_normal((N * N, s))
        A = laplacian_2d(N, sigma)
        out.append(Problem(f"lyap_{i}_N{N}_s{s}", A, None, C1, None, s, "cg", tol, maxit, "fp64",
                           {"N": N, "sigma": sigma}))
    return out
